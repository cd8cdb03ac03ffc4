// Internal data structures of the h2bem library (not part of the C ABI).
//
// The matrix-vector product u2 = M u1 (Eq. denseMat) with the H2 form of M
// (Section "H2-Matrix Compression") is executed as a fixed sequence of
// "passes".  Every pass is a block-sparse product
//
//     out_segment (nrows x r)  (=, +=, atomic +=)  sum_pieces A_piece (nrows x ncols) * in_piece (ncols x r)
//
// over the FP64 workspace (row-major, r values per row).  All matrices a
// matvec reads are packed into one byte arena in the exact order in which the
// passes consume them, so that every pass streams one contiguous range of
// HBM with bulk (TMA) copies.  The host builds the plan once per operator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include "../../include/h2bem.h"

#define H2_MAX_M 5
#define H2_MAX_K 125
#define H2_MAX_LEAF 128
#define H2_MAX_RHS 32
#define H2_MAX_BATCH 16        // operators of one batched product
#define H2_MAX_CHUNK_COLS 128   // input columns of one chunk (shared-memory staging)

// Input columns per chunk of an operator built for up to max_rhs right-hand
// sides: 64 above 8 right-hand sides, so that a stage's input buffer (columns x
// right-hand sides x 8 bytes) stays at 16 KB and three stages fit at 32.
inline int chunk_cols_for(int max_rhs) { return max_rhs > 8 ? 64 : H2_MAX_CHUNK_COLS; }
#define H2_MAX_CHUNK_PIECES 32  // matrices of one chunk (one producer lane each)

namespace h2 {

struct FemData;   // a tetrahedral mesh on the device (h2_fem.cu)
void fem_release(FemData* f);

enum SegMode : int32_t {
    SEG_STORE = 0,      // ws[out_row + i] = sum
    SEG_ATOMIC = 1,     // atomicAdd(ws[out_row + i], sum)
    SEG_FINAL = 2,      // u2[c * N + perm[out_row + i]] = sum
    SEG_ADD = 3,        // ws[out_row + i] += sum (single writer per pass)
    SEG_FINAL_ADD = 4,  // u2[c * N + perm[out_row + i]] += sum (after the near field)
};

// How a stored matrix is laid out and multiplied.  PIECE_F64 / PIECE_F32:
// column-major, CUDA cores.  PIECE_TF32 / PIECE_BF16X3: a tensor-core tile
// (see tc_offset), multiplied by tcgen05.
enum PieceType : int32_t { PIECE_F64 = 0, PIECE_F32 = 1, PIECE_TF32 = 2, PIECE_BF16X3 = 3, PIECE_NODES = 4 };
// PIECE_NODES: a coupling block evaluated in the product (H2_COUPLING_ON_THE_FLY):
// one float4 per column, the source cluster's Chebyshev node minus the target
// box's centre; the target nodes (minus the same centre) come from the
// operator's per-cluster node table.

inline __host__ __device__ bool piece_tc(int type) { return type == PIECE_TF32 || type == PIECE_BF16X3; }
// Stored format of the coupling blocks S_ts of an operator of precision `prec`.
inline int coupling_piece_type(int prec) {
    return prec == H2_FP64 ? PIECE_F64 : prec == H2_FP32 ? PIECE_F32 : prec == H2_TF32X3 ? PIECE_TF32 : PIECE_BF16X3;
}
// Stored format of the transfer matrices E_c.  BF16 hi + lo operators keep
// them in FP32 (the same 4 bytes per entry) on the CUDA cores: a transfer's
// rounding reaches every level above and below it, and 17-bit transfers
// compounded over the tree's 12-16 levels would exceed the 1e-5 budget by
// themselves; they are about a tenth of the far field's entries.
inline int transfer_piece_type(int prec) { return prec == H2_BF16X3 ? PIECE_F32 : coupling_piece_type(prec); }
// Rows of a tensor-core tile (the MMA's M) for a block of `nrows` rows.
inline __host__ __device__ int tc_rows(int nrows) { return nrows <= 64 ? 64 : 128; }
// Columns (the MMA's K) multiplied by one tcgen05.mma.
inline __host__ __device__ int tc_kstep(int type) { return type == PIECE_TF32 ? 8 : 16; }
// Signal units of a finished segment in the dataflow form: one per 16 rows
// (the CUDA-core writer warps each write and signal 16 rows; of a tensor-core
// segment, the four warps that own the TMEM lane quarters signal one unit per
// 16-row group they wrote), whichever pipe multiplied it.
inline __host__ __device__ int segment_writers(int nrows, bool tc) { return (void)tc, (nrows + 15) / 16; }
// Byte offset of entry (i, j) in a tensor-core tile of Mp rows.  The tile is a
// sequence of K slabs (tc_kstep columns each, all rows); a slab holds two
// "core matrices" along K, each Mp/8 groups of 8 rows x 16 bytes, so that
// shared-memory descriptors with a K-direction core stride (LBO) of 16*Mp
// bytes and a row-group stride (SBO) of 128 bytes address it.  BF16X3 slabs
// hold the hi cores followed by the lo cores (`lo` selects them).
inline __host__ __device__ int64_t tc_offset(int type, int Mp, int i, int j, int lo) {
    const int ks = tc_kstep(type);
    const int es = type == PIECE_TF32 ? 4 : 2;
    const int per = 16 / es;
    const int s = j / ks, jj = j % ks;
    const int64_t slab = (int64_t)ks * Mp * 4;   // both types: 4 bytes per entry
    return s * slab + (int64_t)lo * 2 * 16 * Mp + (jj / per) * 16 * Mp + (i / 8) * 128 + (i % 8) * 16 +
           (jj % per) * es;
}

// A contiguous, 16-byte aligned byte range of the arena that one bulk copy
// brings into one shared-memory stage.  It holds whole small blocks or a
// column range of one large block ("pieces").
struct Chunk {
    int64_t src;         // byte offset in the arena
    int32_t bytes;       // multiple of 16
    int32_t piece0;      // first piece (index into the pass's piece array)
    int32_t npieces;
    int32_t ncols;       // input columns of all its pieces (<= H2_MAX_CHUNK_COLS)
    int32_t in_row0;     // input row and type of the first piece (a one-piece chunk
    int32_t type0;       // needs no piece-table read)
};

// One column-major matrix (nrows x ncols, nrows = the segment's) inside a
// stage, multiplied with workspace rows [in_row, in_row + ncols) of the FP64
// workspace (PIECE_F64) or of the FP32 workspace (PIECE_F32).  in_row is a
// multiple of 4, so that the input of a piece (ncols * r values) starts on a
// 16-byte boundary in either workspace.
struct Piece {
    int32_t smem_off;    // byte offset inside the stage (16-byte aligned)
    int32_t in_row;
    int32_t ncols;
    int32_t type;        // PieceType
};

struct Segment {
    int32_t out_row;     // workspace row (or tree position for SEG_FINAL, SEG_FINAL_ADD)
    int32_t nrows;       // <= 128
    int32_t mode;        // SegMode
    int32_t chunk0;      // first chunk
    int32_t nchunks;     // >= 1
    int32_t out_f32;     // 1: the output rows are in the FP32 workspace
};

// Host plan of one pass plus its device copies.
enum PassKind : int32_t {
    PASS_PROLOGUE = 0, PASS_UP_LEAF = 1, PASS_UP_TRANSFER = 2, PASS_COUPLING = 3,
    PASS_DOWN_TRANSFER = 4, PASS_LEAF_NEAR = 5, PASS_LEAF_EXPAND = 6, PASS_FLOW = 7,
    // launches of the split form: the near field on the operator's second
    // stream, the dataflow launch of everything else, the joining addition
    PASS_SPLIT_NEAR = 8, PASS_SPLIT_FAR = 9, PASS_SPLIT_ADD = 10,
};

// One profiled kernel launch: events recorded before and after it on the
// stream it was launched on, with what it computes.
struct ProfLaunch {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int32_t kind = 0, grid = 0, r = 0;
    int64_t bytes = 0, macs = 0;   // matrix bytes read, multiply-adds per right-hand side
};

struct FlowSeg;

struct Pass {
    std::string name;
    int32_t kind = 0;
    std::vector<Segment> seg;
    std::vector<Chunk> chunk;
    std::vector<Piece> piece;
    FlowSeg* d_seg = nullptr;           // uploaded as segments without dependencies
    Chunk* d_chunk = nullptr;
    Piece* d_piece = nullptr;
    int64_t bytes = 0;        // arena bytes streamed by the pass
    int64_t macs = 0;         // multiply-adds per right-hand side
    int grid = 0;             // CTAs of the last launch
};

// One segment of the single-launch dataflow form of the product.  Segments
// are stored in ticket order (a topological order of their dependencies);
// a segment waits until each region in deps[dep0 .. dep0+ndep) has reached
// its expected producer count, and increments `signal` when its output is
// written.  Regions: x-hat of cluster c = c, y-hat of c = nc + c, u2 rows of
// leaf t = 2 nc + t.
struct FlowSeg {
    Segment s;           // chunk0 indexes the flow chunk array
    int32_t signal;      // region completed by this segment (-1: none)
    int32_t dep0, ndep;
    int32_t kind;        // PassKind of the originating pass
    int32_t op;          // operator of a batched launch (0 for one operator)
    int32_t pad;
};

// The dataflow form of one or several operators (one launch): segments in
// ticket order, their chunks and pieces, the regions each segment waits for,
// the number of signals that completes every region, and per operator the
// y-hat rows cleared before the launch.  Regions of operator i are numbered
// after those of operators 0..i-1 (3 n_clusters each).
struct FlowOut {
    std::vector<FlowSeg> seg;
    std::vector<Chunk> chunk;
    std::vector<Piece> piece;
    std::vector<int32_t> deps, expect;
    std::vector<std::vector<int32_t>> zero_rows;
    int nreg = 0;
};

// Where one matrix lives in the arena.
struct MatRef {
    int64_t off = -1;   // byte offset, 16-byte aligned
    int32_t nrows = 0, ncols = 0, type = 0;
};

// An FP64 column-major matrix (rows x cols, leading dimension ld) in a
// device buffer, `off` in doubles.
struct RcSource {
    int64_t off = 0;
    int32_t ld = 0, rows = 0, cols = 0;
};

// The far field of an operator after algebraic recompression
// (h2_params.recompress_eps > 0): the ranks of every cluster's row and
// column bases and, per matrix of the product, where its FP64 values lie
// (d_pool: leaf bases and transfers; d_interp: the couplings, written over
// the interpolation arena they were computed from).  Released after the
// product's arena is assembled.
struct RcResult {
    double* d_pool = nullptr;
    double* d_interp = nullptr;
    std::vector<int32_t> kr, kc;               // per cluster (0: basis unused)
    std::vector<RcSource> Vn, Wn, En, Fn;      // per cluster: leaf bases, transfers (rows, columns)
    std::vector<RcSource> Sn;                  // per far block
    void release_device() {
        if (d_pool) cudaFree(d_pool);
        if (d_interp) cudaFree(d_interp);
        d_pool = d_interp = nullptr;
    }
    ~RcResult() { release_device(); }
};

}  // namespace h2

struct h2_handle {
    int kind = 0;   // 1 geometry, 2 operator, 3 tetrahedral mesh (FEM)
    h2::FemData* fem = nullptr;
    int refcount = 1;
    uint64_t serial = 0;   // unique per handle (keys the batched-launch plans)

    // ---------------- geometry ----------------
    int64_t N = 0, T = 0;
    std::vector<double> xyz;        // host copy, N x 3
    std::vector<int32_t> tri;       // host copy, T x 3
    std::vector<int64_t> adj_ptr;   // node -> triangles (CSR)
    std::vector<int32_t> adj;
    double* d_xyz = nullptr;
    int32_t* d_tri = nullptr;
    int64_t* d_adj_ptr = nullptr;
    int32_t* d_adj = nullptr;
    double* d_psi = nullptr;
    int device = 0;

    // ---------------- operator ----------------
    h2_handle* geom = nullptr;
    h2_params params{};
    int m = 0, k = 0, kp = 0;       // kp = k rounded up to even (workspace row alignment)
    // cluster tree (host), numbered level by level
    int nc = 0, nlevels = 0, nleaves = 0;
    std::vector<int32_t> perm, start, size, parent, child0, child1, level;
    std::vector<double> box;        // 6 per cluster: lo xyz, hi xyz
    std::vector<int32_t> far_t, far_s, near_t, near_s;
    std::vector<char> need_x, need_y, is_src, is_tgt;
    // matrices
    std::vector<h2::MatRef> W, V, Eup, Edown;     // per cluster
    std::vector<h2::MatRef> S;                    // per far block
    std::vector<h2::MatRef> Nb;                   // per near block
    h2::RcResult* rc = nullptr;                   // recompressed far field until the arena holds it
    int64_t arena_bytes = 0;
    unsigned char* d_arena = nullptr;
    int32_t* d_perm = nullptr;
    double* d_box = nullptr;
    // Workspace rows (r values per row; the same numbering in the FP64 and the
    // FP32 workspace): the input in tree order, leaf by leaf, each leaf padded to
    // a multiple of 4 rows (rows [0, row_xhat)); then x-hat and y-hat, kp rows
    // per cluster; then 4 rows of tail padding.  The FP32 workspace exists for
    // FP32 operators, whose far-field vectors (x-hat, y-hat and the copy of the
    // input read by the leaf projections) are FP32.
    int64_t row_xhat = 0, row_yhat = 0, ws_rows = 0;
    std::vector<int32_t> leaf_row;    // first workspace row of each cluster's input (leaves)
    std::vector<int32_t> gather_src;  // per input row: mesh node, or -1 for padding
    int32_t* d_gather_src = nullptr;
    double* d_ws = nullptr;
    float* d_ws32 = nullptr;
    std::vector<int32_t> zero_rows;   // x-hat / y-hat regions accumulated atomically (cleared by the gather)
    int32_t* d_zero_rows = nullptr;
    double* d_io = nullptr;           // device staging for host-pointer calls
    int* d_err = nullptr;             // device error word (bounded waits)
    // passes in launch order
    std::vector<h2::Pass> passes;
    int64_t bytes_streamed = 0, macs = 0;
    int64_t far_bytes = 0, near_bytes = 0, basis_coefficients = 0, near_entries = 0;
    double assemble_seconds = 0.0;
    int stages = 3;                   // shared-memory stages of the pass kernel
    int stage_bytes = 32768;
    int coupling_split = 8;           // far blocks per coupling segment
    int tc_small_r_cuda = 1;          // tensor-core tiles on the CUDA cores at small r (autotuner's switch)
    int chunk_cols = H2_MAX_CHUNK_COLS;   // input columns per chunk (chunk_cols_for(max_rhs))
    double flow_makespan_us = 0.0;    // simulated duration of the dataflow order
    // CUDA graph of one matvec (the gather and the product launches), captured
    // on the second call with the same buffers and r, replayed afterwards
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t capture_stream = nullptr;
    int graph_r = 0;
    const double* graph_u1 = nullptr;
    double* graph_u2 = nullptr;
    int graph_seen = 0;               // direct calls with the current (u1, u2, r)
    int graph_fail = 0;               // capture failed once: launch directly from now on
    // launch configuration chosen by the autotuner (0: defaults)
    int tune_stages = 0;              // shared-memory stages of the segment kernel
    int tune_ctas = 0;                // resident CTAs per SM (cap below the occupancy limit)
    double tune_ms = 0.0;
    int n_launches = 0;
    // single-launch dataflow form
    std::vector<h2::FlowSeg> fseg;
    std::vector<h2::Chunk> fchunk;
    std::vector<h2::Piece> fpiece;
    std::vector<int32_t> fdeps, fexpect, fzero_rows;
    h2::FlowSeg* d_fseg = nullptr;
    h2::Chunk* d_fchunk = nullptr;
    h2::Piece* d_fpiece = nullptr;
    int32_t* d_fdeps = nullptr;
    int32_t* d_fexpect = nullptr;
    int32_t* d_fzero_rows = nullptr;
    int32_t* d_fcnt = nullptr;        // 3 nc region counters + 1 ticket counter
    int flow_grid = 0;                // CTAs of the last dataflow launch
    int nsm = 0;                      // SMs of the device
    int use_flow = 0;
    // split form (reduced precision, r > 8, leaves of at most 64 rows): the
    // FP64 near field in its own launch on a second stream (u2n), beside a
    // dataflow launch of everything else (far field and leaf expansions, added
    // into the cleared u2); one addition joins them
    int has_split = 0;
    int use_split = 1;                // autotuner's switch
    h2::FlowOut split;                // ticket order without the near field
    h2::FlowSeg* d_sseg = nullptr;
    h2::Chunk* d_schunk = nullptr;
    h2::Piece* d_spiece = nullptr;
    int32_t* d_sdeps = nullptr;
    int32_t* d_sexpect = nullptr;
    int32_t* d_szero_rows = nullptr;
    double* d_u2n = nullptr;          // max_rhs x N
    std::vector<std::array<int32_t, 4>> near_units;   // near-field work units: segment, first chunk, chunks
    int4* d_near_units = nullptr;
    float4* d_nodes = nullptr;        // evaluated coupling: kp Chebyshev nodes per cluster, minus its box's centre
    // paired near field (h2_near_field H2_NEAR_F32PAIR, split form only):
    // the near pass's arena bytes [near_lo, near_hi) again, every FP64 value
    // as two FP32 words hi, lo; the input rows as pairs, laid out like d_ws
    float2* d_near_pair = nullptr;
    int64_t near_lo = 0, near_hi = 0;
    float2* d_wsp = nullptr;
    cudaStream_t near_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // per-pass timing with CUDA events (profiling aid, off by default)
    int prof_enabled = 0;
    std::vector<std::vector<h2::ProfLaunch>> prof_calls;   // launches of each profiled call
    std::vector<cudaEvent_t> prof_pool;
};

namespace h2 {
// Cost model of one CTA of the segment kernel, used to order the dataflow
// form (list scheduling on `workers` simulated CTAs).
struct FlowModel {
    int workers = 304;           // resident CTAs of the launch
    int r = 1;                   // right-hand sides the order is tuned for
    double seg_ns = 1500.0;      // fixed cost of a segment (dependency signal, reduction, write)
    double chunk_ns = 150.0;     // fixed cost of a chunk (barrier, input staging)
    double f64_per_ns = 2.07;    // FP64 multiply-adds per ns of one CTA
    double f32_per_ns = 130.0;   // FP32 multiply-adds per ns of one CTA
    double bytes_per_ns = 22.0;  // HBM bytes per ns of one CTA
};

// host-side builders (h2_host.cpp)
int validate_mesh(const double* xyz, int64_t N, const int32_t* tri, int64_t T,
                  std::vector<int64_t>& adj_ptr, std::vector<int32_t>& adj);
void build_cluster_tree(h2_handle* op);
void build_block_partition(h2_handle* op);
void gauss_legendre_unit(int q, std::vector<double>& x, std::vector<double>& w);
void build_plan(h2_handle* op);   // arena layout + passes (h2_plan.cpp)
double build_flow(h2_handle* op, const FlowModel& fm);   // dataflow order (h2_plan.cpp)
double build_flow_multi(const std::vector<h2_handle*>& ops, const FlowModel& fm, FlowOut& out,
                        bool without_near = false);
bool split_possible(const h2_handle* op);   // the split form applies to this operator
int build_split(h2_handle* op);             // its ticket order (host)

// device-side assembly and matvec (h2_assemble.cu, h2_matvec.cu)
int geometry_device_setup(h2_handle* g, cudaStream_t s);
int assemble_device(h2_handle* op, cudaStream_t s);
int assemble_interp_far(h2_handle* op, cudaStream_t s, unsigned char* arena);
// Algebraic recompression of the far field on the device (h2_recompress.cu):
// fills op->rc (ranks and FP64 matrices); build_plan then lays out the
// product with those ranks and assemble_device stores them.
int recompress_device(h2_handle* op, cudaStream_t s);
int upload_plan(h2_handle* op);
int matvec_device(h2_handle* op, const double* u1, double* u2, int r, cudaStream_t s);
void release_graph(h2_handle* op);
void release_profile(h2_handle* op);
int read_profile(h2_handle* op, std::vector<ProfLaunch>& launches, std::vector<double>& ms, int& ncalls);
size_t pass_smem_bytes(const h2_handle* op, int rt);
int flow_model(h2_handle* op, FlowModel& fm);   // CTAs and rates of the device
// One persistent launch over several operators (h2_matvec_batched).
int matvec_batched(h2_handle* const* ops, int n, const double* const* u1, double* const* u2, const int32_t* r,
                   cudaStream_t s);
void drop_batch_plans(uint64_t serial);   // forget the plans that use an operator
int autotune(h2_handle* op, int r, cudaStream_t s, h2_tuning_t* out);
}  // namespace h2

// Returns H2_ERR_OOM or H2_ERR_CUDA from the enclosing function when a CUDA
// call fails; the message names the error, the call and its source line.
#define H2_CUDA_TRY(call)                                        \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) {                                 \
            h2::set_cuda_error(e_, #call, __FILE__, __LINE__);   \
            return e_ == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA; \
        }                                                        \
    } while (0)

namespace h2 {
void set_last_error(const char* msg);
void set_cuda_error(cudaError_t e, const char* call, const char* file, int line);
}
