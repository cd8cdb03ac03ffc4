// h2_plan_check: the execution plan of h2_assemble built on the host alone
// (no device work), and the invariants the product kernels rely on, checked
// independently of the builders that made them.
//
// The cluster tree, the block partition (Section "H2-Matrix Compression":
// admissible blocks and exact near blocks), the passes of the product (upward
// leaf projection and transfers, coupling, downward transfers, near field,
// leaf expansion) and the dataflow ticket order (with and without the near
// field, as the split form uses it, and the merged order of a batched launch)
// come from the same host code as in h2_assemble and h2_matvec_batched.  The
// checks:
//   * every chunk is a legal bulk copy (16-byte aligned source and size, at
//     most one stage, its pieces inside it, input rows on 4-row boundaries,
//     one piece type per chunk, one accumulator kind per segment);
//   * the ticket order is a topological order: every producer of a region a
//     segment waits for holds an earlier ticket (a persistent CTA that waits
//     only for earlier tickets cannot deadlock);
//   * every region's expected signal count equals the writer signals of its
//     producers, and every region a segment waits for either has producers
//     or expects nothing.
#include <cstring>
#include <new>
#include <vector>

#include "h2_internal.h"

namespace {

int check_chunks(const h2_handle& op, const std::vector<h2::Chunk>& chunks, const std::vector<h2::Piece>& pieces) {
    int bad = 0;
    for (const h2::Chunk& c : chunks) {
        bool ok = c.src % 16 == 0 && c.bytes % 16 == 0 && c.bytes > 0 && c.bytes <= op.stage_bytes &&
                  c.npieces >= 1 && c.npieces <= H2_MAX_CHUNK_PIECES && c.ncols >= 1 && c.ncols <= op.chunk_cols &&
                  c.src + c.bytes <= op.arena_bytes && c.piece0 >= 0 &&
                  (size_t)c.piece0 + (size_t)c.npieces <= pieces.size();
        if (ok) {
            int cols = 0;
            for (int q = 0; q < c.npieces && ok; ++q) {
                const h2::Piece& p = pieces[(size_t)c.piece0 + q];
                ok = p.ncols >= 1 && p.in_row >= 0 && p.in_row % 4 == 0 && p.smem_off % 16 == 0 && p.smem_off >= 0 &&
                     p.smem_off < c.bytes && (int64_t)p.in_row + p.ncols <= op.ws_rows - 4 && p.type == c.type0;
                cols += p.ncols;
            }
            ok = ok && cols == c.ncols && pieces[(size_t)c.piece0].in_row == c.in_row0;
        }
        bad += ok ? 0 : 1;
    }
    return bad;
}

int check_flow(const h2_handle& op, const h2::FlowOut& f) {
    int bad = check_chunks(op, f.chunk, f.piece);
    const size_t n = f.seg.size();
    std::vector<int64_t> last_producer(f.nreg, -1), expect(f.nreg, 0), producers(f.nreg, 0);
    for (size_t i = 0; i < n; ++i) {
        const h2::FlowSeg& s = f.seg[i];
        const h2::Segment& g = s.s;
        if (g.nchunks < 1 || g.nrows < 1 || g.nrows > H2_MAX_LEAF || g.chunk0 < 0 ||
            (size_t)g.chunk0 + (size_t)g.nchunks > f.chunk.size()) {
            ++bad;
            continue;
        }
        const bool tc0 = h2::piece_tc(f.chunk[(size_t)g.chunk0].type0);
        for (int q = 0; q < g.nchunks; ++q) {
            const int t = f.chunk[(size_t)g.chunk0 + q].type0;
            if (h2::piece_tc(t) != tc0 || (g.out_f32 && t == h2::PIECE_F64)) ++bad;
        }
        if (s.signal >= f.nreg || (s.signal < 0 && g.mode != h2::SEG_FINAL_ADD)) ++bad;
        if (s.signal >= 0 && s.signal < f.nreg) {
            last_producer[s.signal] = (int64_t)i;
            expect[s.signal] += h2::segment_writers(g.nrows, tc0);
            producers[s.signal]++;
        }
        if (s.dep0 < 0 || s.ndep < 0 || (size_t)s.dep0 + (size_t)s.ndep > f.deps.size()) ++bad;
    }
    if (f.expect.size() != (size_t)f.nreg) return bad + 1;
    for (int r = 0; r < f.nreg; ++r)
        if (expect[r] != f.expect[r]) ++bad;
    for (size_t i = 0; i < n; ++i) {
        const h2::FlowSeg& s = f.seg[i];
        if (s.dep0 < 0 || (size_t)s.dep0 + (size_t)s.ndep > f.deps.size()) continue;
        for (int q = 0; q < s.ndep; ++q) {
            const int32_t d = f.deps[(size_t)s.dep0 + q];
            if (d < 0 || d >= f.nreg) {
                ++bad;
                continue;
            }
            // every producer of d before this segment: the last one is enough
            if (last_producer[d] >= (int64_t)i) ++bad;
            if (producers[d] == 0 && f.expect[d] != 0) ++bad;
        }
    }
    return bad;
}

}  // namespace

int h2_plan_check(const double* xyz, int64_t n_vertices, const int32_t* tri, int64_t n_triangles,
                  const h2_params* p_in, int32_t workers, h2_plan_report_t* out) {
    if (!xyz || !tri || !out || workers < 1) return H2_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    h2_params p;
    if (p_in) p = *p_in;
    else h2_default_params(&p);
    if (p.m < 1 || p.m > H2_MAX_M || p.leaf < 1 || p.leaf > H2_MAX_LEAF || !(p.eta > 0.0) ||
        !(p.box_inflation > 0.0) || p.box_inflation > 1.0 || p.max_rhs < 1 || p.max_rhs > H2_MAX_RHS ||
        p.precision < H2_FP64 || p.precision > H2_BF16X3 ||
        (p.coupling != H2_COUPLING_STORED && p.coupling != H2_COUPLING_ON_THE_FLY) ||
        (p.coupling == H2_COUPLING_ON_THE_FLY && p.precision != H2_FP32) ||
        (p.schedule != H2_SCHEDULE_FLOW && p.schedule != H2_SCHEDULE_LEVELS) || (p.autotune != 0 && p.autotune != 1) ||
        (p.near_field != H2_NEAR_FP64 && p.near_field != H2_NEAR_F32PAIR))
        return H2_ERR_INVALID_ARG;
    h2_handle* geom = new (std::nothrow) h2_handle();
    h2_handle* op = new (std::nothrow) h2_handle();
    if (!geom || !op) {
        delete geom;
        delete op;
        return H2_ERR_OOM;
    }
    int rc = h2::validate_mesh(xyz, n_vertices, tri, n_triangles, geom->adj_ptr, geom->adj);
    if (rc == H2_OK) {
        geom->kind = 1;
        geom->N = n_vertices;
        geom->T = n_triangles;
        geom->xyz.assign(xyz, xyz + 3 * n_vertices);
        geom->tri.assign(tri, tri + 3 * n_triangles);
        op->kind = 2;
        op->geom = geom;
        op->params = p;
        op->m = p.m;
        op->k = p.m * p.m * p.m;
        op->kp = (op->k + 3) / 4 * 4;
        h2::build_cluster_tree(op);
        h2::build_block_partition(op);
        h2::build_plan(op);
        h2::FlowModel fm;
        fm.workers = workers;
        fm.r = p.max_rhs;
        h2::FlowOut full, split;
        out->makespan_us = h2::build_flow_multi({op}, fm, full, false);
        const double ms_split = h2::build_flow_multi({op}, fm, split, true);
        int bad = 0;
        for (const h2::Pass& q : op->passes) bad += check_chunks(*op, q.chunk, q.piece);
        if (out->makespan_us < 0.0) ++bad;
        else bad += check_flow(*op, full);
        if (ms_split >= 0.0) bad += check_flow(*op, split);
        // the merged order of a batched launch (here the operator twice: the
        // second copy's regions follow the first's)
        h2::FlowOut twice;
        if (h2::build_flow_multi({op, op}, fm, twice, false) < 0.0) ++bad;
        else {
            bad += check_flow(*op, twice);
            if (twice.nreg != 2 * full.nreg || twice.seg.size() != 2 * full.seg.size()) ++bad;
        }
        out->n_clusters = op->nc;
        out->n_levels = op->nlevels;
        out->n_far_blocks = (int64_t)op->far_t.size();
        out->n_near_blocks = (int64_t)op->near_t.size();
        out->n_segments = (int64_t)full.seg.size();
        out->n_chunks = (int64_t)full.chunk.size();
        out->n_regions = full.nreg;
        out->n_split_segments = ms_split >= 0.0 ? (int64_t)split.seg.size() : -1;
        out->split_makespan_us = ms_split;
        out->bytes_streamed = op->bytes_streamed;
        out->violations = bad;
    }
    delete op;
    delete geom;
    return rc;
}
