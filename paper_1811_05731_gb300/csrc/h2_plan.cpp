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
        auto close = [&]() {
            if (cur.src >= 0 && cur.npieces > 0) p.chunk.push_back(cur);
            cur = Chunk{};
            cur.src = -1;
        };
        for (const MatSpec& m : s.mats) {
            const int es = esize(m.type);
            const int64_t mbytes = round16((int64_t)s.nrows * m.ncols * es);
            m.ref->off = arena;
            m.ref->nrows = s.nrows;
            m.ref->ncols = m.ncols;
            m.ref->type = m.type;
            p.macs += (int64_t)s.nrows * m.ncols;
            if (mbytes <= stage) {
                if (cur.src >= 0 && (arena + mbytes - cur.src) > stage) close();
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
                cur.bytes = (int32_t)(arena + mbytes - cur.src);
            } else {
                close();
                const int step = es == 8 ? 2 : 4;   // keeps every piece a multiple of 16 bytes
                int cols = (int)(stage / ((int64_t)s.nrows * es));
                cols = std::max(step, cols / step * step);
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
    // F: leaf expansion + near field + diagonal, scattered to u2
    {
        std::vector<std::vector<int32_t>> near_by_t(nc);
        for (size_t b = 0; b < op->near_t.size(); ++b) near_by_t[op->near_t[b]].push_back((int32_t)b);
        std::vector<SegSpec> segs;
        for (int t = 0; t < nc; ++t) {
            if (op->child0[t] >= 0) continue;
            SegSpec s;
            s.out_row = op->start[t];
            s.nrows = op->size[t];
            s.mode = SEG_FINAL;
            if (op->need_y[t]) {
                s.mats.push_back({&op->V[t], k, P, yrow(t)});
                s.bytes += (int64_t)op->size[t] * k * (P == PIECE_F64 ? 2 : 1);
            }
            for (int32_t b : near_by_t[t]) {
                const int32_t sc = op->near_s[b];
                s.mats.push_back({&op->Nb[b], op->size[sc], PIECE_F64, op->start[sc]});
                s.bytes += 2LL * op->size[t] * op->size[sc];
            }
            segs.push_back(s);
        }
        emit_pass(op, "leaf_near", PASS_LEAF_NEAR, segs, arena);
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

}  // namespace h2
