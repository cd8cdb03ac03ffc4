// Execution plan of the H2 matrix-vector product (arXiv:1811.05731, Section
// "H2-Matrix Compression": nested cluster bases, k x k coupling matrices per
// admissible block, exact near-field blocks).
//
// The product y = M x is evaluated in passes:
//   U0      x-hat_s = W_s^T x|_s                    leaves s that need x-hat
//   U(l)    x-hat_t = sum_children E_c^T x-hat_c    level l = L-2 .. 0 (upward)
//   C       y-hat_t += S_ts x-hat_s                 all admissible blocks
//   D(l)    y-hat_c (+)= E_c y-hat_parent           level l = 1 .. L-1 (downward)
//   F       y|_t = V_t y-hat_t + sum_s N_ts x|_s    leaves (near field incl. the
//                                                   solid-angle diagonal), written
//                                                   to u2 in mesh node order
// Every matrix is stored column-major (rows = outputs) at a 16-byte aligned
// offset of one arena, in the order in which the passes read them.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "h2_internal.h"

namespace h2 {

namespace {

inline int64_t round16(int64_t b) { return (b + 15) & ~(int64_t)15; }

struct MatSpec {
    MatRef* ref;        // where to record the arena offset
    int32_t ncols;
    int32_t type;
    int32_t in_row;
};

struct SegSpec {
    int32_t out_row, nrows, mode;
    std::vector<MatSpec> mats;
    int64_t bytes = 0;
};

int esize(int type) { return type == PIECE_F64 ? 8 : 4; }

// Lays out the matrices of one pass in the arena and cuts them into chunks.
void emit_pass(h2_handle* op, const char* name, int32_t kind, std::vector<SegSpec>& segs,
               int64_t& arena) {
    if (segs.empty()) return;
    // longest segments first: round-robin assignment then approximates LPT
    std::stable_sort(segs.begin(), segs.end(),
                     [](const SegSpec& a, const SegSpec& b) { return a.bytes > b.bytes; });
    Pass p;
    p.name = name;
    p.kind = kind;
    const int64_t stage = op->stage_bytes;
    for (const SegSpec& s : segs) {
        Segment sg{};
        sg.out_row = s.out_row;
        sg.nrows = s.nrows;
        sg.mode = s.mode;
        sg.chunk0 = (int32_t)p.chunk.size();
        Chunk cur{};
        cur.src = -1;
        int cur_cols = 0;
        auto close = [&]() {
            if (cur.src >= 0 && cur.npieces > 0) p.chunk.push_back(cur);
            cur = Chunk{};
            cur.src = -1;
            cur_cols = 0;
        };
        for (const MatSpec& m : s.mats) {
            const int es = esize(m.type);
            const int64_t mbytes = round16((int64_t)s.nrows * m.ncols * es);
            m.ref->off = arena;
            m.ref->nrows = s.nrows;
            m.ref->ncols = m.ncols;
            m.ref->type = m.type;
            p.macs += (int64_t)s.nrows * m.ncols;
            if (mbytes <= stage && m.ncols <= H2_MAX_CHUNK_COLS) {
                if (cur.src >= 0 && ((arena + mbytes - cur.src) > stage ||
                                     cur_cols + m.ncols > H2_MAX_CHUNK_COLS))
                    close();
                if (cur.src < 0) {
                    cur.src = arena;
                    cur.piece0 = (int32_t)p.piece.size();
                    cur.npieces = 0;
                }
                Piece pc{};
                pc.smem_off = (int32_t)(arena - cur.src);
                pc.in_row = m.in_row;
                pc.ncols = m.ncols;
                pc.type = m.type;
                p.piece.push_back(pc);
                cur.npieces++;
                cur_cols += m.ncols;
                cur.bytes = (int32_t)(arena + mbytes - cur.src);
            } else {
                close();
                const int step = es == 8 ? 2 : 4;   // keeps every piece a multiple of 16 bytes
                int cols = (int)(stage / ((int64_t)s.nrows * es));
                cols = std::max(step, std::min(cols, H2_MAX_CHUNK_COLS) / step * step);
                for (int c0 = 0; c0 < m.ncols; c0 += cols) {
                    const int cc = std::min(cols, m.ncols - c0);
                    Chunk ch{};
                    ch.src = arena + (int64_t)c0 * s.nrows * es;
                    ch.bytes = (int32_t)round16((int64_t)cc * s.nrows * es);
                    ch.piece0 = (int32_t)p.piece.size();
                    ch.npieces = 1;
                    Piece pc{};
                    pc.smem_off = 0;
                    pc.in_row = m.in_row + c0;
                    pc.ncols = cc;
                    pc.type = m.type;
                    p.piece.push_back(pc);
                    p.chunk.push_back(ch);
                }
            }
            arena += mbytes;
            p.bytes += mbytes;
        }
        close();
        sg.nchunks = (int32_t)p.chunk.size() - sg.chunk0;
        p.seg.push_back(sg);
    }
    op->passes.push_back(std::move(p));
}

}  // namespace

void build_plan(h2_handle* op) {
    const int nc = op->nc;
    const int k = op->k;
    const int kp = op->kp;
    const int P = op->params.precision == H2_FP32 ? PIECE_F32 : PIECE_F64;
    const int64_t N = op->geom->N;

    op->is_src.assign(nc, 0);
    op->is_tgt.assign(nc, 0);
    for (size_t b = 0; b < op->far_t.size(); ++b) {
        op->is_tgt[op->far_t[b]] = 1;
        op->is_src[op->far_s[b]] = 1;
    }
    // x-hat_c is needed where c is a source or lies below one; y-hat_c where
    // c is a target or lies below one (clusters are numbered parents first).
    op->need_x.assign(nc, 0);
    op->need_y.assign(nc, 0);
    for (int c = 0; c < nc; ++c) {
        const int p = op->parent[c];
        op->need_x[c] = op->is_src[c] || (p >= 0 && op->need_x[p]);
        op->need_y[c] = op->is_tgt[c] || (p >= 0 && op->need_y[p]);
    }

    op->row_xhat = (N + 1) / 2 * 2;
    op->row_yhat = op->row_xhat + (int64_t)nc * kp;
    op->ws_rows = op->row_yhat + (int64_t)nc * kp + 2;
    auto xrow = [&](int c) { return (int32_t)(op->row_xhat + (int64_t)c * kp); };
    auto yrow = [&](int c) { return (int32_t)(op->row_yhat + (int64_t)c * kp); };

    op->W.assign(nc, MatRef{});
    op->V.assign(nc, MatRef{});
    op->Eup.assign(nc, MatRef{});
    op->Edown.assign(nc, MatRef{});
    op->S.assign(op->far_t.size(), MatRef{});
    op->Nb.assign(op->near_t.size(), MatRef{});
    op->passes.clear();
    int64_t arena = 0;

    // U0: leaf projections
    {
        std::vector<SegSpec> segs;
        for (int c = 0; c < nc; ++c) {
            if (op->child0[c] >= 0 || !op->need_x[c]) continue;
            SegSpec s;
            s.out_row = xrow(c);
            s.nrows = k;
            s.mode = SEG_STORE;
            s.mats.push_back({&op->W[c], op->size[c], P, op->start[c]});
            s.bytes = (int64_t)k * op->size[c];
            segs.push_back(s);
        }
        emit_pass(op, "up_leaf", PASS_UP_LEAF, segs, arena);
    }
    // U(l): transfers towards the root
    for (int l = op->nlevels - 2; l >= 0; --l) {
        std::vector<SegSpec> segs;
        for (int c = 0; c < nc; ++c) {
            if (op->level[c] != l || op->child0[c] < 0 || !op->need_x[c]) continue;
            SegSpec s;
            s.out_row = xrow(c);
            s.nrows = k;
            s.mode = SEG_STORE;
            for (int ch : {op->child0[c], op->child1[c]})
                s.mats.push_back({&op->Eup[ch], k, P, xrow(ch)});
            s.bytes = 2LL * k * k;
            segs.push_back(s);
        }
        emit_pass(op, "up_transfer", PASS_UP_TRANSFER, segs, arena);
    }
    // C: coupling, grouped by target and split into groups of at most `split`
    // blocks (atomic accumulation into the cleared y-hat)
    {
        std::vector<std::vector<int32_t>> by_t(nc);
        for (size_t b = 0; b < op->far_t.size(); ++b) by_t[op->far_t[b]].push_back((int32_t)b);
        const int64_t nfar = (int64_t)op->far_t.size();
        const int split = 8;
        std::vector<SegSpec> segs;
        op->zero_rows.clear();
        for (int t = 0; t < nc; ++t) {
            if (by_t[t].empty()) continue;
            op->zero_rows.push_back(yrow(t));
            for (size_t g0 = 0; g0 < by_t[t].size(); g0 += split) {
                SegSpec s;
                s.out_row = yrow(t);
                s.nrows = k;
                s.mode = SEG_ATOMIC;
                for (size_t g = g0; g < std::min(by_t[t].size(), g0 + split); ++g) {
                    const int32_t b = by_t[t][g];
                    s.mats.push_back({&op->S[b], k, P, xrow(op->far_s[b])});
                    s.bytes += (int64_t)k * k;
                }
                segs.push_back(s);
            }
        }
        (void)nfar;
        emit_pass(op, "coupling", PASS_COUPLING, segs, arena);
    }
    // D(l): transfers towards the leaves
    for (int l = 1; l < op->nlevels; ++l) {
        std::vector<SegSpec> segs;
        for (int c = 0; c < nc; ++c) {
            if (op->level[c] != l) continue;
            const int p = op->parent[c];
            if (p < 0 || !op->need_y[p]) continue;
            SegSpec s;
            s.out_row = yrow(c);
            s.nrows = k;
            s.mode = op->is_tgt[c] ? SEG_ADD : SEG_STORE;
            s.mats.push_back({&op->Edown[c], k, P, yrow(p)});
            s.bytes = (int64_t)k * k;
            segs.push_back(s);
        }
        emit_pass(op, "down_transfer", PASS_DOWN_TRANSFER, segs, arena);
    }
    // F1: near field + diagonal, scattered to u2 (overwrites u2)
    std::vector<std::vector<int32_t>> near_by_t(nc);
    for (size_t b = 0; b < op->near_t.size(); ++b) near_by_t[op->near_t[b]].push_back((int32_t)b);
    {
        std::vector<SegSpec> segs;
        for (int t = 0; t < nc; ++t) {
            if (op->child0[t] >= 0) continue;
            SegSpec s;
            s.out_row = op->start[t];
            s.nrows = op->size[t];
            s.mode = SEG_FINAL;
            for (int32_t b : near_by_t[t]) {
                const int32_t sc = op->near_s[b];
                s.mats.push_back({&op->Nb[b], op->size[sc], PIECE_F64, op->start[sc]});
                s.bytes += 2LL * op->size[t] * op->size[sc];
            }
            segs.push_back(s);
        }
        emit_pass(op, "leaf_near", PASS_LEAF_NEAR, segs, arena);
    }
    // F2: leaf expansion y|_t += V_t y-hat_t (adds to u2)
    {
        std::vector<SegSpec> segs;
        for (int t = 0; t < nc; ++t) {
            if (op->child0[t] >= 0 || !op->need_y[t]) continue;
            SegSpec s;
            s.out_row = op->start[t];
            s.nrows = op->size[t];
            s.mode = SEG_FINAL_ADD;
            s.mats.push_back({&op->V[t], k, P, yrow(t)});
            s.bytes = (int64_t)op->size[t] * k * (P == PIECE_F64 ? 2 : 1);
            segs.push_back(s);
        }
        emit_pass(op, "leaf_expand", PASS_LEAF_EXPAND, segs, arena);
    }
    op->arena_bytes = arena;

    op->bytes_streamed = 0;
    op->macs = 0;
    for (const Pass& p : op->passes) {
        op->bytes_streamed += p.bytes;
        op->macs += p.macs;
    }
    op->near_bytes = 0;
    op->near_entries = 0;
    for (size_t b = 0; b < op->near_t.size(); ++b) {
        op->near_entries += (int64_t)op->size[op->near_t[b]] * op->size[op->near_s[b]];
        op->near_bytes += round16((int64_t)op->size[op->near_t[b]] * op->size[op->near_s[b]] * 8);
    }
    op->far_bytes = op->arena_bytes - op->near_bytes;
    op->basis_coefficients = 0;
    for (int c = 0; c < nc; ++c) {
        for (const MatRef* r : {&op->W[c], &op->V[c], &op->Eup[c], &op->Edown[c]})
            if (r->off >= 0) op->basis_coefficients += (int64_t)r->nrows * r->ncols;
    }
}

// Single-launch dataflow form: every segment of every pass in one list, in
// a topological order of the data dependencies that also puts the critical
// path (upward chain -> coupling of the upper targets -> downward chain)
// early and uses the near field (no dependencies) to fill the upward phase.
void build_flow(h2_handle* op) {
    const int nc = op->nc;
    const int kp = op->kp;
    const int64_t N = op->geom->N;
    op->fseg.clear();
    op->fchunk.clear();
    op->fpiece.clear();
    op->fdeps.clear();
    op->fexpect.assign((size_t)3 * nc, 0);
    op->fzero_rows.clear();
    op->use_flow = 0;

    auto cluster_of_row = [&](int64_t row, int& region_base) -> int {
        if (row < op->row_xhat) { region_base = -1; return -1; }
        if (row < op->row_yhat) { region_base = 0; return (int)((row - op->row_xhat) / kp); }
        region_base = nc;
        return (int)((row - op->row_yhat) / kp);
    };
    std::vector<int32_t> leaf_at(N + 1, -1);
    for (int c = 0; c < nc; ++c)
        if (op->child0[c] < 0) leaf_at[op->start[c]] = c;

    struct Item { FlowSeg fs; std::vector<int32_t> deps; int level; };
    std::vector<Item> up_leaf, near, vexp_all;
    std::vector<std::vector<Item>> up_lv, coup_lv(op->nlevels), down_lv(op->nlevels + 1),
        vexp_lv(op->nlevels);
    std::vector<char> zero(nc, 0);

    for (const Pass& p : op->passes) {
        std::vector<Item> items;
        for (const Segment& sg0 : p.seg) {
            Item it{};
            it.fs.s = sg0;
            it.fs.kind = p.kind;
            it.fs.s.chunk0 = (int32_t)op->fchunk.size();
            for (int q = 0; q < sg0.nchunks; ++q) {
                Chunk ch = p.chunk[(size_t)sg0.chunk0 + q];
                const int32_t pbase = (int32_t)op->fpiece.size();
                for (int u = 0; u < ch.npieces; ++u) {
                    const Piece pc = p.piece[(size_t)ch.piece0 + u];
                    op->fpiece.push_back(pc);
                    int rb;
                    const int c = cluster_of_row(pc.in_row, rb);
                    if (c >= 0) {
                        const int32_t reg = rb + c;
                        if (std::find(it.deps.begin(), it.deps.end(), reg) == it.deps.end())
                            it.deps.push_back(reg);
                    }
                }
                ch.piece0 = pbase;
                op->fchunk.push_back(ch);
            }
            // output region and level
            int c = -1;
            if (sg0.mode == SEG_FINAL || sg0.mode == SEG_FINAL_ADD) {
                c = leaf_at[sg0.out_row];
                if (sg0.mode == SEG_FINAL) it.fs.signal = 2 * nc + c;
                else {
                    it.fs.signal = -1;
                    it.deps.push_back(2 * nc + c);   // after the near field of the leaf
                }
            } else {
                int rb;
                c = cluster_of_row(sg0.out_row, rb);
                it.fs.signal = rb + c;
                if (rb == nc) {   // y-hat: every producer accumulates atomically
                    it.fs.s.mode = SEG_ATOMIC;
                    zero[c] = 1;
                }
            }
            it.level = op->level[c];
            if (it.fs.signal >= 0) op->fexpect[it.fs.signal]++;
            items.push_back(std::move(it));
        }
        switch (p.kind) {
            case PASS_UP_LEAF: for (auto& i : items) up_leaf.push_back(std::move(i)); break;
            case PASS_UP_TRANSFER: up_lv.push_back(std::move(items)); break;
            case PASS_COUPLING: for (auto& i : items) coup_lv[i.level].push_back(std::move(i)); break;
            case PASS_DOWN_TRANSFER: for (auto& i : items) down_lv[i.level].push_back(std::move(i)); break;
            case PASS_LEAF_NEAR: for (auto& i : items) near.push_back(std::move(i)); break;
            case PASS_LEAF_EXPAND: for (auto& i : items) vexp_lv[i.level].push_back(std::move(i)); break;
            default: return;
        }
    }
    // ticket order
    std::vector<Item*> order;
    for (auto& i : up_leaf) order.push_back(&i);
    const size_t nslices = std::max<size_t>(1, up_lv.size());
    size_t nq = 0;
    for (size_t l = 0; l < nslices; ++l) {
        if (l < up_lv.size())
            for (auto& i : up_lv[l]) order.push_back(&i);
        const size_t end = near.size() * (l + 1) / nslices;
        for (; nq < end; ++nq) order.push_back(&near[nq]);
    }
    for (; nq < near.size(); ++nq) order.push_back(&near[nq]);
    for (int l = 0; l < op->nlevels; ++l) {
        for (auto& i : coup_lv[l]) order.push_back(&i);
        if (l + 1 <= op->nlevels)
            for (auto& i : down_lv[l + 1]) order.push_back(&i);
        for (auto& i : vexp_lv[l]) order.push_back(&i);
    }
    // every dependency must be produced by earlier tickets only
    std::vector<int32_t> last_producer((size_t)3 * nc, -1);
    for (size_t t = 0; t < order.size(); ++t)
        if (order[t]->fs.signal >= 0) last_producer[order[t]->fs.signal] = (int32_t)t;
    for (size_t t = 0; t < order.size(); ++t)
        for (int32_t d : order[t]->deps)
            if (last_producer[d] < 0 || last_producer[d] >= (int32_t)t) return;   // keep level-wise launches
    for (Item* it : order) {
        it->fs.dep0 = (int32_t)op->fdeps.size();
        it->fs.ndep = (int32_t)it->deps.size();
        for (int32_t d : it->deps) op->fdeps.push_back(d);
        op->fseg.push_back(it->fs);
    }
    for (int c = 0; c < nc; ++c)
        if (zero[c]) op->fzero_rows.push_back((int32_t)(op->row_yhat + (int64_t)c * kp));
    op->use_flow = 1;
}

}  // namespace h2
