// Execution plan of the H2 matrix-vector product (arXiv:1811.05731, Section
// "H2-Matrix Compression": nested cluster bases, k x k coupling matrices per
// admissible block, exact near-field blocks).
//
// The product y = M x is evaluated in passes:
//   U0      x-hat_s = W_s^T x|_s                    leaves s that need x-hat
//   U(l)    x-hat_t += E_c^T x-hat_c                level l = L-2 .. 0 (upward), one
//                                                   segment per child c of t, so that
//                                                   each starts as soon as x-hat_c is
//                                                   complete (two atomic additions to
//                                                   the cleared x-hat_t: exact order
//                                                   independence)
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
#include <queue>
#include <utility>

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
        sg.out_f32 = op->params.precision != H2_FP64 && s.mode != SEG_FINAL && s.mode != SEG_FINAL_ADD;
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
            const bool tc = piece_tc(m.type);
            const int es = esize(m.type);
            // tensor-core tiles: Mp rows x Kp columns, 4 bytes per entry (TF32,
            // or BF16 hi + lo); column-major blocks otherwise
            const int Mp = tc_rows(s.nrows);
            const int kcols = tc ? (m.ncols + tc_kstep(m.type) - 1) / tc_kstep(m.type) * tc_kstep(m.type) : m.ncols;
            // (evaluated coupling blocks: one float4 source node per column)
            const int64_t col_bytes = tc ? (int64_t)Mp * 4 : m.type == PIECE_NODES ? 16 : (int64_t)s.nrows * es;
            const int64_t mbytes = round16(col_bytes * kcols);
            m.ref->off = arena;
            m.ref->nrows = s.nrows;
            m.ref->ncols = m.ncols;
            m.ref->type = m.type;
            p.macs += (int64_t)s.nrows * m.ncols;
            if (mbytes <= stage && kcols <= op->chunk_cols) {
                if (cur.src >= 0 && ((arena + mbytes - cur.src) > stage ||
                                     cur_cols + m.ncols > op->chunk_cols ||
                                     cur.npieces >= H2_MAX_CHUNK_PIECES))
                    close();
                if (cur.src < 0) {
                    cur.src = arena;
                    cur.piece0 = (int32_t)p.piece.size();
                    cur.npieces = 0;
                    cur.in_row0 = m.in_row;
                    cur.type0 = m.type;
                }
                Piece pc{};
                pc.smem_off = (int32_t)(arena - cur.src);
                pc.in_row = m.in_row;
                pc.ncols = m.ncols;
                pc.type = m.type;
                p.piece.push_back(pc);
                cur.npieces++;
                cur_cols += m.ncols;
                cur.ncols = cur_cols;
                cur.bytes = (int32_t)(arena + mbytes - cur.src);
            } else {
                close();
                // split into column ranges (whole K slabs for tensor-core tiles);
                // every range starts on a multiple of 4 columns, so its input
                // rows stay 16-byte aligned
                const int step = tc ? tc_kstep(m.type) : 4;
                int cols = (int)(stage / col_bytes);
                cols = std::max(step, std::min(cols, op->chunk_cols) / step * step);
                for (int c0 = 0; c0 < kcols; c0 += cols) {
                    const int cc = std::min(cols, kcols - c0);
                    const int real = std::max(0, std::min(cc, m.ncols - c0));   // input columns
                    if (real == 0) break;
                    Chunk ch{};
                    ch.src = arena + (int64_t)c0 * col_bytes;
                    ch.bytes = (int32_t)round16((int64_t)cc * col_bytes);
                    ch.piece0 = (int32_t)p.piece.size();
                    ch.npieces = 1;
                    ch.ncols = real;
                    ch.in_row0 = m.in_row + c0;
                    ch.type0 = m.type;
                    Piece pc{};
                    pc.smem_off = 0;
                    pc.in_row = m.in_row + c0;
                    pc.ncols = real;
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
    op->chunk_cols = chunk_cols_for(op->params.max_rhs);
    const int nc = op->nc;
    const int k = op->k;
    const int kp = op->kp;
    // leaf bases (P), transfer matrices (PT) and coupling blocks (PC) per precision
    const int prec = op->params.precision;
    const int P = prec == H2_FP64 ? PIECE_F64 : PIECE_F32;
    const int PT = transfer_piece_type(prec);   // transfers E_c
    const int PC = coupling_piece_type(prec);   // coupling blocks S_ts
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

    // input rows: leaf by leaf in tree order, each leaf padded to 4 rows
    op->leaf_row.assign(nc, -1);
    op->gather_src.clear();
    std::vector<int32_t> leaves;
    for (int c = 0; c < nc; ++c)
        if (op->child0[c] < 0) leaves.push_back(c);
    std::sort(leaves.begin(), leaves.end(), [&](int32_t x, int32_t y) { return op->start[x] < op->start[y]; });
    for (int32_t c : leaves) {
        op->leaf_row[c] = (int32_t)op->gather_src.size();
        for (int a = 0; a < op->size[c]; ++a) op->gather_src.push_back(op->perm[op->start[c] + a]);
        while (op->gather_src.size() % 4) op->gather_src.push_back(-1);
    }
    (void)N;
    op->row_xhat = (int64_t)op->gather_src.size();
    op->row_yhat = op->row_xhat + (int64_t)nc * kp;
    op->ws_rows = op->row_yhat + (int64_t)nc * kp + 4;
    auto xrow = [&](int c) { return (int32_t)(op->row_xhat + (int64_t)c * kp); };
    auto yrow = [&](int c) { return (int32_t)(op->row_yhat + (int64_t)c * kp); };
    // ranks of the cluster bases: k everywhere for the interpolation operator,
    // the recompression's ranks otherwise (rows of y-hat_c and of x-hat_c; the
    // workspace slots keep their kp rows)
    auto krow = [&](int c) { return op->rc ? op->rc->kr[c] : k; };
    auto kcol = [&](int c) { return op->rc ? op->rc->kc[c] : k; };

    op->zero_rows.clear();   // workspace regions accumulated atomically, cleared by the gather
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
            if (kcol(c) <= 0) continue;
            SegSpec s;
            s.out_row = xrow(c);
            s.nrows = kcol(c);
            s.mode = SEG_STORE;
            s.mats.push_back({&op->W[c], op->size[c], P, op->leaf_row[c]});
            s.bytes = (int64_t)kcol(c) * op->size[c];
            segs.push_back(s);
        }
        emit_pass(op, "up_leaf", PASS_UP_LEAF, segs, arena);
    }
    // U(l): transfers towards the root, one segment per child
    for (int l = op->nlevels - 2; l >= 0; --l) {
        std::vector<SegSpec> segs;
        for (int c = 0; c < nc; ++c) {
            if (op->level[c] != l || op->child0[c] < 0 || !op->need_x[c]) continue;
            op->zero_rows.push_back(xrow(c));
            for (int ch : {op->child0[c], op->child1[c]}) {
                if (kcol(c) <= 0 || kcol(ch) <= 0) continue;
                SegSpec s;
                s.out_row = xrow(c);
                s.nrows = kcol(c);
                s.mode = SEG_ATOMIC;
                s.mats.push_back({&op->Eup[ch], kcol(ch), PT, xrow(ch)});
                s.bytes = (int64_t)kcol(c) * kcol(ch);
                segs.push_back(s);
            }
        }
        emit_pass(op, "up_transfer", PASS_UP_TRANSFER, segs, arena);
    }
    // C: coupling, grouped by target and split into groups of at most `split`
    // blocks (atomic accumulation into the cleared y-hat); within a target the
    // blocks are ordered by the level of their source, deepest first (the
    // order in which the sources' x-hat complete), so that a group does not
    // hold early sources back behind a late one
    {
        std::vector<std::vector<int32_t>> by_t(nc);
        for (size_t b = 0; b < op->far_t.size(); ++b) by_t[op->far_t[b]].push_back((int32_t)b);
        for (auto& v : by_t)
            std::stable_sort(v.begin(), v.end(), [&](int32_t x, int32_t y) {
                return op->level[op->far_s[x]] > op->level[op->far_s[y]];
            });
        const int64_t nfar = (int64_t)op->far_t.size();
        const int split = op->coupling_split;
        const int PS = op->params.coupling == H2_COUPLING_ON_THE_FLY ? PIECE_NODES : PC;   // coupling blocks
        std::vector<SegSpec> segs;
        for (int t = 0; t < nc; ++t) {
            if (by_t[t].empty()) continue;
            op->zero_rows.push_back(yrow(t));
            for (size_t g0 = 0; g0 < by_t[t].size(); g0 += split) {
                SegSpec s;
                s.out_row = yrow(t);
                s.nrows = krow(t);
                s.mode = SEG_ATOMIC;
                for (size_t g = g0; g < std::min(by_t[t].size(), g0 + split); ++g) {
                    const int32_t b = by_t[t][g];
                    if (kcol(op->far_s[b]) <= 0) continue;
                    s.mats.push_back({&op->S[b], kcol(op->far_s[b]), PS, xrow(op->far_s[b])});
                    s.bytes += (int64_t)krow(t) * kcol(op->far_s[b]);
                }
                if (s.nrows > 0 && !s.mats.empty()) segs.push_back(s);
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
            if (krow(c) <= 0 || krow(p) <= 0) continue;
            SegSpec s;
            s.out_row = yrow(c);
            s.nrows = krow(c);
            s.mode = op->is_tgt[c] ? SEG_ADD : SEG_STORE;
            s.mats.push_back({&op->Edown[c], krow(p), PT, yrow(p)});
            s.bytes = (int64_t)krow(c) * krow(p);
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
                s.mats.push_back({&op->Nb[b], op->size[sc], PIECE_F64, op->leaf_row[sc]});
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
            if (krow(t) <= 0) continue;
            SegSpec s;
            s.out_row = op->start[t];
            s.nrows = op->size[t];
            s.mode = SEG_FINAL_ADD;
            s.mats.push_back({&op->V[t], krow(t), P, yrow(t)});
            s.bytes = (int64_t)op->size[t] * krow(t) * (P == PIECE_F64 ? 2 : 1);
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

// Single-launch dataflow form: every segment of every pass in one list of
// "tickets" that the CTAs of one persistent launch take in order.  A segment
// may only follow the producers of the regions it reads, and a CTA that
// takes a segment whose inputs are not complete waits for them, so the
// order decides how much time is lost waiting.  It is chosen by simulating
// `workers` CTAs on the host: each free CTA takes, among the segments whose
// producers are all placed, the one with the longest remaining path to the
// end of the product (critical path first) among those whose inputs will be
// complete by then, else the one whose inputs complete first.  Segment cost:
// a fixed overhead plus the larger of its FP64 multiply-adds, FP32
// multiply-adds and matrix bytes at one CTA's share of the SM and HBM rates.
// Returns the simulated makespan in microseconds (or -1 if the dataflow form
// could not be built; the level-wise launches are used then).
// without_near: the near-field segments are left out (the split form runs
// them in a launch of their own) and the leaf expansions add into u2 without
// waiting for them.
double build_flow_multi(const std::vector<h2_handle*>& ops, const FlowModel& fm, FlowOut& out, bool without_near) {
    out = FlowOut{};
    struct Item {
        FlowSeg fs;
        std::vector<int32_t> deps;
        double cost = 0.0, blevel = 0.0;
    };
    std::vector<Item> items;
    const double r = std::max(1, fm.r);
    int reg_base = 0;
    std::vector<int32_t> producers;   // per region
    out.zero_rows.resize(ops.size());
    for (size_t oi = 0; oi < ops.size(); ++oi) {
        h2_handle* op = ops[oi];
        const int nc = op->nc;
        const int kp = op->kp;
        const int64_t N = op->geom->N;
        auto cluster_of_row = [&](int64_t row, int& region_base) -> int {
            if (row < op->row_xhat) { region_base = -1; return -1; }
            if (row < op->row_yhat) { region_base = 0; return (int)((row - op->row_xhat) / kp); }
            region_base = nc;
            return (int)((row - op->row_yhat) / kp);
        };
        std::vector<int32_t> leaf_at(N + 1, -1);
        for (int c = 0; c < nc; ++c)
            if (op->child0[c] < 0) leaf_at[op->start[c]] = c;
        std::vector<char> zero(2 * nc, 0);   // x-hat (c) and y-hat (nc + c) regions written atomically
        producers.resize((size_t)reg_base + 3 * nc, 0);
        for (const Pass& p : op->passes) {
            if (without_near && p.kind == PASS_LEAF_NEAR) continue;
            for (const Segment& sg0 : p.seg) {
                Item it{};
                it.fs.s = sg0;
                it.fs.kind = p.kind;
                it.fs.op = (int32_t)oi;
                it.fs.s.chunk0 = (int32_t)out.chunk.size();
                double mac64 = 0.0, mac32 = 0.0, bytes = 0.0;
                for (int q = 0; q < sg0.nchunks; ++q) {
                    Chunk ch = p.chunk[(size_t)sg0.chunk0 + q];
                    const int32_t pbase = (int32_t)out.piece.size();
                    bytes += ch.bytes;
                    for (int u = 0; u < ch.npieces; ++u) {
                        const Piece pc = p.piece[(size_t)ch.piece0 + u];
                        out.piece.push_back(pc);
                        (pc.type == PIECE_F64 ? mac64 : mac32) += (double)sg0.nrows * pc.ncols * r;
                        int rb;
                        const int c = cluster_of_row(pc.in_row, rb);
                        if (c >= 0) {
                            const int32_t reg = reg_base + rb + c;
                            if (std::find(it.deps.begin(), it.deps.end(), reg) == it.deps.end())
                                it.deps.push_back(reg);
                        }
                    }
                    ch.piece0 = pbase;
                    out.chunk.push_back(ch);
                }
                it.cost = fm.seg_ns + fm.chunk_ns * sg0.nchunks +
                          std::max({mac64 / fm.f64_per_ns, mac32 / fm.f32_per_ns, bytes / fm.bytes_per_ns});
                if (sg0.mode == SEG_FINAL || sg0.mode == SEG_FINAL_ADD) {
                    const int c = leaf_at[sg0.out_row];
                    if (sg0.mode == SEG_FINAL) it.fs.signal = reg_base + 2 * nc + c;
                    else {
                        it.fs.signal = -1;
                        if (!without_near) it.deps.push_back(reg_base + 2 * nc + c);   // after the near field of the leaf
                    }
                } else {
                    int rb;
                    const int c = cluster_of_row(sg0.out_row, rb);
                    it.fs.signal = reg_base + rb + c;
                    if (rb == nc) {   // y-hat: every producer accumulates atomically
                        it.fs.s.mode = SEG_ATOMIC;
                        zero[nc + c] = 1;
                    } else if (it.fs.s.mode == SEG_ATOMIC) {
                        zero[c] = 1;
                    }
                }
                if (it.fs.signal >= 0) producers[it.fs.signal]++;
                items.push_back(std::move(it));
            }
        }
        for (int c = 0; c < nc; ++c)
            if (zero[c]) out.zero_rows[oi].push_back((int32_t)(op->row_xhat + (int64_t)c * kp));
        for (int c = 0; c < nc; ++c)
            if (zero[nc + c]) out.zero_rows[oi].push_back((int32_t)(op->row_yhat + (int64_t)c * kp));
        reg_base += 3 * nc;
    }
    const int nreg = reg_base;
    const int n = (int)items.size();
    // consumers of every region
    std::vector<std::vector<int32_t>> consumers(nreg);
    for (int i = 0; i < n; ++i)
        for (int32_t d : items[i].deps) consumers[d].push_back(i);
    // longest path to the end: every operator's passes are listed in a
    // topological order, so one sweep in reverse settles every consumer before
    // its producers
    std::vector<double> reg_blevel(nreg, 0.0);
    for (int i = n - 1; i >= 0; --i) {
        Item& it = items[i];
        it.blevel = it.cost + (it.fs.signal >= 0 ? reg_blevel[it.fs.signal] : 0.0);
        for (int32_t d : it.deps) reg_blevel[d] = std::max(reg_blevel[d], it.blevel);
    }
    // list scheduling on `workers` simulated CTAs
    std::vector<int32_t> reg_left(producers);
    std::vector<double> reg_done(nreg, 0.0);
    std::vector<int32_t> deps_left(n);
    std::vector<double> ready_at(n, 0.0);
    using Cand = std::pair<double, int32_t>;
    std::priority_queue<Cand> ready;                                            // by b-level
    std::priority_queue<Cand, std::vector<Cand>, std::greater<Cand>> pending;   // by ready time
    for (int i = 0; i < n; ++i) {
        deps_left[i] = (int32_t)items[i].deps.size();
        for (int32_t d : items[i].deps)
            if (reg_left[d] == 0) deps_left[i]--;   // region without producers: nothing to wait for
        if (deps_left[i] == 0) pending.push({0.0, i});
    }
    std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
    for (int w = 0; w < std::max(1, fm.workers); ++w) free_at.push(0.0);
    std::vector<int32_t> order;
    order.reserve(n);
    double makespan = 0.0;
    while ((int)order.size() < n) {
        const double t = free_at.top();
        free_at.pop();
        while (!pending.empty() && pending.top().first <= t) {
            ready.push({items[pending.top().second].blevel, pending.top().second});
            pending.pop();
        }
        int32_t pick;
        if (!ready.empty()) {
            pick = ready.top().second;
            ready.pop();
        } else if (!pending.empty()) {
            pick = pending.top().second;
            pending.pop();
        } else {
            return -1.0;   // a region that never completes: no dataflow form
        }
        const double start = std::max(t, ready_at[pick]);
        const double fin = start + items[pick].cost;
        makespan = std::max(makespan, fin);
        free_at.push(fin);
        order.push_back(pick);
        const int32_t sig = items[pick].fs.signal;
        if (sig >= 0) {
            reg_done[sig] = std::max(reg_done[sig], fin);
            if (--reg_left[sig] == 0) {
                for (int32_t c : consumers[sig]) {
                    ready_at[c] = std::max(ready_at[c], reg_done[sig]);
                    if (--deps_left[c] == 0) pending.push({ready_at[c], c});
                }
            }
        }
    }
    // every writer warp of the kernel signals a finished segment
    out.expect.assign(nreg, 0);
    for (const Item& it : items)
        if (it.fs.signal >= 0)
            out.expect[it.fs.signal] += segment_writers(it.fs.s.nrows, piece_tc(out.chunk[it.fs.s.chunk0].type0));
    for (int32_t i : order) {
        Item& it = items[i];
        it.fs.dep0 = (int32_t)out.deps.size();
        it.fs.ndep = (int32_t)it.deps.size();
        for (int32_t d : it.deps) out.deps.push_back(d);
        out.seg.push_back(it.fs);
    }
    out.nreg = nreg;
    return makespan * 1e-3;
}

double build_flow(h2_handle* op, const FlowModel& fm) {
    FlowOut o;
    op->use_flow = 0;
    const double ms = build_flow_multi({op}, fm, o);
    if (ms < 0.0) return ms;   // keep the level-wise launches
    op->fseg = std::move(o.seg);
    op->fchunk = std::move(o.chunk);
    op->fpiece = std::move(o.piece);
    op->fdeps = std::move(o.deps);
    op->fexpect = std::move(o.expect);
    op->fzero_rows = std::move(o.zero_rows[0]);
    op->use_flow = 1;
    return ms;
}

}  // namespace h2
