// The H2 matrix-vector product u2 = M u1 (arXiv:1811.05731, Eq. denseMat;
// Section "H2-Matrix Compression") on one GPU.
//
// The product is a set of "segments": each sums column-major matrices times
// workspace vectors into rows of the workspace (x-hat, y-hat) or of u2.  The
// matrices lie in one arena in the order in which segments consume them and
// are streamed into a ring of shared-memory stages by one elected thread with
// bulk TMA copies (cp.async.bulk completing on mbarrier transaction counts).
// All threads compute from shared memory: thread (row, g) accumulates row
// `row` over the columns congruent to g modulo G = 256 / nrows, and the G
// partial sums are added in shared memory at the end of the segment.
//
// Two schedules execute the same segments:
//  * k_flow (default): ONE persistent launch.  CTAs take segments through an
//    atomic ticket in a topological order; before computing, a segment waits
//    (bounded) until the regions it reads (x-hat of a cluster, y-hat of a
//    cluster, the near-field rows of a leaf) have all their producers done;
//    after writing, it signals its own region.  The bulk-copy ring keeps
//    prefetching the next segments' matrices while a segment waits.
//  * k_pass: one launch per pass (upward leaf, each upward level, coupling,
//    each downward level, near field, leaf expansion).
//
// FP64 pieces accumulate in FP64 (two independent FMA chains per thread for
// one right-hand side).  FP32 pieces (far field of an FP32 operator) multiply
// and accumulate in FP32 within a piece and add the piece's sum to the FP64
// accumulator; the workspace and u2 are FP64.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "h2_internal.h"

namespace h2 {

namespace {

constexpr int kConsumers = 256;                          // compute threads (8 warps)
constexpr int kBlock = kConsumers + 32;                  // + one producer warp
constexpr int kMaxStages = 4;
constexpr int kMaxChunkCols = H2_MAX_CHUNK_COLS;         // input columns staged per chunk
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s bound on every device-side wait

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the phase did not complete within kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (true) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (now_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// What the producer warp publishes with every staged chunk.
struct StageDesc {
    int32_t seg;       // segment index (-1: this CTA has no more work)
    int32_t last;      // 1 if the chunk is the last of its segment
    int32_t npieces;
    int32_t f32;       // 1 if the chunk's matrices and inputs are FP32
    int32_t out_row, nrows, mode, signal;
    int32_t out_f32;   // 1 if the segment's output rows are FP32
    int32_t ptype;     // PieceType of the chunk's matrices
    int32_t cbytes;    // bytes of the chunk's matrices in the stage
    int32_t op;        // operator (batched launches)
    int32_t pad;
};

// One matrix of a staged chunk, as the consumers read it.
struct SPiece {
    int32_t smem_off;   // byte offset of the matrix inside the stage
    int32_t in_row;     // first workspace row of its input
    int32_t ncols;
    int32_t xoff;       // byte offset of its input inside the stage's input buffer
};

// What a segment of operator `op` needs of its operator.
struct OpCtx {
    const unsigned char* arena;
    double* ws;                // FP64 workspace
    float* ws32;               // FP32 workspace (reduced-precision operators)
    double* u2;
    const int32_t* perm;
    int64_t N;
    int r;
    int kp;                    // cluster vector rows (evaluated coupling: the node table's stride)
    const float4* nodes;       // evaluated coupling: Chebyshev nodes minus the box centre, per cluster
    int64_t row_yhat;          // first y-hat row of the workspace
};

struct KArgs {
    const FlowSeg* seg;        // segments (dataflow form: in ticket order)
    const Chunk* chunk;
    const Piece* piece;
    const int32_t* deps;       // dataflow form only
    const int32_t* expect;     // dataflow form only
    int32_t* cnt;              // dataflow form: region counters, ticket counter at [nreg]
    int* err;
    int nseg;
    int nreg;
    int r;                     // largest r of the launch's operators
    int stages;
    int stage_bytes;
    int xin_bytes;             // input buffer of one stage (xin_bytes(RT); FP32 rows: xin_bytes_f32(RT))
    int tc;                    // the operator has tensor-core segments
    int tc_alo_bytes;          // shared memory for the TF32 lo parts of a chunk
    int tc_b_bytes;            // shared memory for the B operand (all its parts) of a chunk
    int tc_parts;              // most vector parts of a launch's tiles (3: BF16 hi, mid, lo; 2: TF32 hi, lo)
    int tc_sets;               // operand sets (2: the next chunk is prepared while the tensor core works)
    int tc_cols;               // TMEM columns per CTA (power of 2, at most 512 / resident CTAs per SM)
    int tc_nacc;               // accumulators of the A_hi products (K steps round-robin)
    int tc_ncorr;              // accumulators of the A_lo correction products (round-robin)
    int tc_np;                 // columns of one vector part: right-hand sides rounded up to 16
    int tc_cuda;               // 1: tensor-core tiles multiplied on the CUDA cores (small r)
    int nops;                  // operators of the launch (several: a batched product)
    OpCtx ctx[H2_MAX_BATCH];
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Bounded wait that also gives up as soon as another thread of the CTA set
// the abort flag.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (true) {
        for (int i = 0; i < 16; ++i)
            if (mbar_try(bar, parity)) return true;
        if (*abort_flag || now_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void signal_region(int32_t* p, int n = 1) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(n) : "memory");
}

// The producer warp's source of segments (lane 0).  FLOW: the global ticket
// counter (topological order); otherwise segments blockIdx.x,
// blockIdx.x + gridDim.x, ... of one pass.  Returns -1 when none is left.
template <bool FLOW>
__device__ __forceinline__ int take_segment(const KArgs& a, int& k) {
    const int t = FLOW ? atomicAdd(a.cnt + a.nreg, 1) : (int)blockIdx.x + (k++) * (int)gridDim.x;
    return t < a.nseg ? t : -1;
}

// Bounded wait (lane 0 of the producer) until every region segment `sg`
// reads has all its producers done.  False on timeout or abort.
__device__ bool deps_wait(const KArgs& a, const FlowSeg& F, volatile int* abort_flag) {
    for (int d = F.dep0; d < F.dep0 + F.ndep; ++d) {
        const int reg = a.deps[d];
        const int want = a.expect[reg];
        if (ld_acquire(a.cnt + reg) >= want) continue;
        const unsigned long long t0 = now_ns();
        while (ld_acquire(a.cnt + reg) < want) {
            if (*abort_flag || ld_acquire(a.err) != 0 || now_ns() - t0 > kWaitNs) return false;
            __nanosleep(32);
        }
    }
    return true;
}

// Bytes of the staged input of one piece: ncols rows of r values, rounded up
// to 16 (the bulk copy may read up to 3 values past the piece's rows; every
// workspace region is followed by padding or another region).
__device__ __forceinline__ int input_bytes(int ncols, int r, bool f32) {
    return ((ncols * r * (f32 ? 4 : 8)) + 15) & ~15;
}

// Issues the bulk copies of a chunk's inputs (lane p copies piece p's
// workspace rows, which are contiguous) into the stage's input buffer; they
// complete on the stage's `full` barrier.  Workspace values written by other
// CTAs of the launch were published with release/acquire on the region
// counters; the proxy fence orders them before these async-proxy reads.
__device__ __forceinline__ void issue_inputs(const OpCtx& c, const SPiece* pc, int npieces, bool f32,
                                             unsigned char* xin, uint64_t* bar, int lane) {
    if (lane < npieces) {
        const SPiece P = pc[lane];
        const int bytes = input_bytes(P.ncols, c.r, f32);
        const unsigned char* src = f32 ? reinterpret_cast<const unsigned char*>(c.ws32 + (int64_t)P.in_row * c.r)
                                       : reinterpret_cast<const unsigned char*>(c.ws + (int64_t)P.in_row * c.r);
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(xin + P.xoff)),
            "l"(src), "r"(bytes), "r"(smem_addr(bar))
            : "memory");
    }
}

// Error-free FP32 addition (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Multiplies the pieces of one staged chunk into the thread's accumulators.
// FP64 chunks add into `acc`.  FP32 chunks (far-field matrices, leaf bases)
// stay on the FP32 pipe, which GB300 runs at 64 times the FP64 rate: the
// chunk's products are summed in FP32; in a segment with FP32 output
// (`packed`) each accumulator register pair holds a compensated FP32 sum
// (hi word: sum, lo word: the TwoSum error terms), which the segment end
// converts once; otherwise the chunk's sum is added to the FP64 accumulator.
// With r == RT the inputs of one column are read as 16-byte vectors, and the
// FP32 products of two right-hand sides go through one packed FMA
// (__ffma2_rn, each half rounded as fmaf): the FP32 far field at r = 16 is
// bound by instruction issue, and the packed form halves its FMA
// instructions.  At RT = 1 the FP64 products run in two chains, acc[0] and
// acc1, which persist over the segment's chunks and meet at its end.
template <int RT>
__device__ __forceinline__ void consume_chunk(const unsigned char* stage, const SPiece* pieces, int npieces,
                                              bool f32, const unsigned char* xin, int r, int nrows, int row,
                                              int g, int G, bool packed, double (&acc)[RT], double& acc1) {
    if (!f32) {
        for (int p = 0; p < npieces; ++p) {
            const SPiece P = pieces[p];
            const int nc = P.ncols;
            const double* A = reinterpret_cast<const double*>(stage + P.smem_off) + row;
            const double* x = reinterpret_cast<const double*>(xin + P.xoff);
            if (RT == 1) {
                double a0 = acc[0], a1 = acc1;
                int col = g;
#pragma unroll 4
                for (; col + G < nc; col += 2 * G) {
                    a0 = fma(A[col * nrows], x[col], a0);
                    a1 = fma(A[(col + G) * nrows], x[col + G], a1);
                }
                if (col < nc) a0 = fma(A[col * nrows], x[col], a0);
                acc[0] = a0;
                acc1 = a1;
            } else if (r == RT) {   // 16-byte aligned rows of RT values
#pragma unroll 2
                for (int col = g; col < nc; col += G) {
                    const double v = A[col * nrows];
                    const double2* x2 = reinterpret_cast<const double2*>(x + col * RT);
#pragma unroll
                    for (int c = 0; c < RT / 2; ++c) {
                        const double2 xv = x2[c];
                        acc[2 * c] = fma(v, xv.x, acc[2 * c]);
                        acc[2 * c + 1] = fma(v, xv.y, acc[2 * c + 1]);
                    }
                }
            } else {
#pragma unroll 2
                for (int col = g; col < nc; col += G) {
                    const double v = A[col * nrows];
#pragma unroll
                    for (int c = 0; c < RT; ++c)
                        if (c < r) acc[c] = fma(v, x[col * r + c], acc[c]);
                }
            }
        }
        return;
    }
    // the chunk's FP32 sums, right-hand sides 2c and 2c + 1 in acc2[c]
    float2 acc2[(RT + 1) / 2];
#pragma unroll
    for (int c = 0; c < (RT + 1) / 2; ++c) acc2[c] = make_float2(0.0f, 0.0f);
    for (int p = 0; p < npieces; ++p) {
        const SPiece P = pieces[p];
        const int nc = P.ncols;
        const float* A = reinterpret_cast<const float*>(stage + P.smem_off) + row;
        const float* x = reinterpret_cast<const float*>(xin + P.xoff);
        if (RT == 1) {
            float a0 = 0.0f, a1 = 0.0f;
            int col = g;
#pragma unroll 4
            for (; col + G < nc; col += 2 * G) {
                a0 = fmaf(A[col * nrows], x[col], a0);
                a1 = fmaf(A[(col + G) * nrows], x[col + G], a1);
            }
            if (col < nc) a0 = fmaf(A[col * nrows], x[col], a0);
            acc2[0].x += a0 + a1;
        } else if (RT % 4 == 0 && r == RT) {   // 16-byte aligned rows of RT values
#pragma unroll 2
            for (int col = g; col < nc; col += G) {
                const float v = A[col * nrows];
                const float2 v2 = make_float2(v, v);
                const float4* x4 = reinterpret_cast<const float4*>(x + col * RT);
#pragma unroll
                for (int c = 0; c < RT / 4; ++c) {
                    const float4 xv = x4[c];
                    acc2[2 * c] = __ffma2_rn(v2, make_float2(xv.x, xv.y), acc2[2 * c]);
                    acc2[2 * c + 1] = __ffma2_rn(v2, make_float2(xv.z, xv.w), acc2[2 * c + 1]);
                }
            }
        } else {
#pragma unroll 2
            for (int col = g; col < nc; col += G) {
                const float v = A[col * nrows];
#pragma unroll
                for (int c = 0; c < RT; ++c) {
                    if (c >= r) break;
                    float& s = (c & 1) ? acc2[c >> 1].y : acc2[c >> 1].x;
                    s = fmaf(v, x[col * r + c], s);
                }
            }
        }
    }
    if (packed) {
#pragma unroll
        for (int c = 0; c < RT; ++c) {
            float s, e;
            two_sum(__int_as_float(__double2hiint(acc[c])), (c & 1) ? acc2[c >> 1].y : acc2[c >> 1].x, s, e);
            const float l = __int_as_float(__double2loint(acc[c])) + e;
            acc[c] = __hiloint2double(__float_as_int(s), __float_as_int(l));
        }
    } else {
#pragma unroll
        for (int c = 0; c < RT; ++c) acc[c] += (double)((c & 1) ? acc2[c >> 1].y : acc2[c >> 1].x);
    }
}

// Coupling blocks evaluated in the product (H2_COUPLING_ON_THE_FLY): each
// staged column is a source node y (minus the target box's centre), the
// thread's row a target node x (minus the same centre), and the block entry
// S(x, y) = 1 / (4 pi |x - y|) is formed in FP32 (rsqrtf) and applied to the
// column's inputs; sums as for FP32 chunks (packed compensated pair).
constexpr float kInv4Pi = 0.0795774715459476679f;

template <int RT>
__device__ __forceinline__ void consume_nodes(const unsigned char* stage, const SPiece* pieces, int npieces,
                                              const unsigned char* xin, int r, float4 xt, int g, int G,
                                              double (&acc)[RT]) {
    float acc32[RT];
#pragma unroll
    for (int c = 0; c < RT; ++c) acc32[c] = 0.0f;
    for (int p = 0; p < npieces; ++p) {
        const SPiece P = pieces[p];
        const float4* Y = reinterpret_cast<const float4*>(stage + P.smem_off);
        const float* x = reinterpret_cast<const float*>(xin + P.xoff);
#pragma unroll 2
        for (int col = g; col < P.ncols; col += G) {
            const float4 y = Y[col];
            const float dx = xt.x - y.x, dy = xt.y - y.y, dz = xt.z - y.z;
            const float sv = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) * kInv4Pi;
            if (RT % 4 == 0 && r == RT) {
                const float4* x4 = reinterpret_cast<const float4*>(x + col * RT);
#pragma unroll
                for (int c = 0; c < RT / 4; ++c) {
                    const float4 xv = x4[c];
                    acc32[4 * c] = fmaf(sv, xv.x, acc32[4 * c]);
                    acc32[4 * c + 1] = fmaf(sv, xv.y, acc32[4 * c + 1]);
                    acc32[4 * c + 2] = fmaf(sv, xv.z, acc32[4 * c + 2]);
                    acc32[4 * c + 3] = fmaf(sv, xv.w, acc32[4 * c + 3]);
                }
            } else {
#pragma unroll
                for (int c = 0; c < RT; ++c)
                    if (c < r) acc32[c] = fmaf(sv, x[col * r + c], acc32[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < RT; ++c) {
        float s, e;
        two_sum(__int_as_float(__double2hiint(acc[c])), acc32[c], s, e);
        const float l = __int_as_float(__double2loint(acc[c])) + e;
        acc[c] = __hiloint2double(__float_as_int(s), __float_as_int(l));
    }
}

// Largest r at which tensor-core tiles may be multiplied on the CUDA cores.
constexpr int kTcCudaMaxRT = 4;

// Tensor-core tiles (3xTF32, BF16 hi + lo) multiplied on the CUDA cores, for
// few right-hand sides, where one tcgen05.mma of N = 8..16 columns costs as much
// as one of 128 and the products are bound by the bytes streamed: the same
// stored values (TF32 tiles: FP32 entries; BF16: hi + lo, exact in FP32),
// FP32 FMAs, the chunk's sums added to the packed compensated FP32 pair (the
// segments of these tiles have FP32 outputs).  Thread (row, g) takes the
// 16-byte core rows g, g+G, ... of its row (4 TF32 or 8 BF16 columns each,
// see tc_offset), so that a warp reads 512 contiguous bytes per core row.
template <int RT>
__device__ __forceinline__ void consume_tc_tiles(const unsigned char* stage, const SPiece* pieces, int npieces,
                                                 int type, const unsigned char* xin, int r, int nrows, int row,
                                                 int g, int G, double (&acc)[RT]) {
    const int Mp = tc_rows(nrows);
    const int ks = tc_kstep(type);
    const bool bf = type == PIECE_BF16X3;
    const int per = bf ? 8 : 4;
    const int64_t slab = (int64_t)ks * Mp * 4;
    const int rowoff = (row >> 3) * 128 + (row & 7) * 16;
    float acc32[RT];
#pragma unroll
    for (int c = 0; c < RT; ++c) acc32[c] = 0.0f;
    for (int p = 0; p < npieces; ++p) {
        const SPiece P = pieces[p];
        const unsigned char* T = stage + P.smem_off + rowoff;
        const float* x = reinterpret_cast<const float*>(xin + P.xoff);
        const int units = 2 * ((P.ncols + ks - 1) / ks);   // core rows of this row: two per K slab
        for (int u = g; u < units; u += G) {
            const int j0 = (u >> 1) * ks + (u & 1) * per;
            if (j0 >= P.ncols) continue;
            const unsigned char* src = T + (u >> 1) * slab + (u & 1) * 16 * Mp;
            float a[8];
            if (bf) {
                const uint4 h = *reinterpret_cast<const uint4*>(src);
                const uint4 l = *reinterpret_cast<const uint4*>(src + 32 * Mp);
                const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {   // bf16 -> f32: the 16 bits as the high half
                    a[2 * e] = __uint_as_float(hw[e] << 16) + __uint_as_float(lw[e] << 16);
                    a[2 * e + 1] = __uint_as_float(hw[e] & 0xFFFF0000u) + __uint_as_float(lw[e] & 0xFFFF0000u);
                }
            } else {
                const float4 v = *reinterpret_cast<const float4*>(src);
                a[0] = v.x;
                a[1] = v.y;
                a[2] = v.z;
                a[3] = v.w;
            }
            const int ne = P.ncols - j0 < per ? P.ncols - j0 : per;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                if (e >= per || e >= ne) break;
                const float* xj = x + (j0 + e) * r;
#pragma unroll
                for (int c = 0; c < RT; ++c)
                    if (c < r) acc32[c] = fmaf(a[e], xj[c], acc32[c]);
            }
        }
    }
#pragma unroll
    for (int c = 0; c < RT; ++c) {
        float s, e;
        two_sum(__int_as_float(__double2hiint(acc[c])), acc32[c], s, e);
        const float l = __int_as_float(__double2loint(acc[c])) + e;
        acc[c] = __hiloint2double(__float_as_int(s), __float_as_int(l));
    }
}

// Sum of the G packed compensated FP32 partial sums of one output value
// (see consume_chunk), in FP32 with TwoSum: no FP64 arithmetic.
__device__ __forceinline__ float packed_sum(const double* red, int stride, int G) {
    float s = 0.0f, e = 0.0f;
    for (int g2 = 0; g2 < G; ++g2) {
        const double d = red[g2 * stride];
        float t, u;
        two_sum(s, __int_as_float(__double2hiint(d)), t, u);
        s = t;
        e += u + __int_as_float(__double2loint(d));
    }
    return s + e;
}

// Writer warps of a segment: warp w < writer_warps(nrows) adds the G partial
// sums of rows 16w .. 16w+15 (lanes l and l+16: row 16w + l, the first and the
// second half of the right-hand sides c0 .. c0+cn-1), stored in `red` with
// stride `rs` per thread, and writes them; up to all eight consumer warps share
// the writing, the others go on with the next chunk.  One right-hand side
// (cn == 1 always): rows 32w .. 32w+31, one per lane, and the writer warps
// past the rows only signal.
__host__ __device__ constexpr int writer_warps(int nrows) { return (nrows + 15) / 16; }

__device__ __forceinline__ void write_segment(const StageDesc& D, const double* red, int rs, int c0, int cn, int r,
                                              int G, double* ws, float* ws32, double* u2,
                                              const int32_t* __restrict__ perm, int64_t N) {
    const int nrows = D.nrows;
    const int lane = threadIdx.x & 31;
    const bool one = rs == 1;
    const int rr = one ? (int)threadIdx.x : 16 * (threadIdx.x >> 5) + (lane & 15);   // writer warps only
    if (rr >= nrows) return;
    const int ch = (cn + 1) >> 1;
    const int cb = one || lane < 16 ? 0 : ch, ce = one ? cn : lane < 16 ? ch : cn;
    const bool fin = D.mode == SEG_FINAL || D.mode == SEG_FINAL_ADD;
    const int64_t orow = fin ? (int64_t)perm[D.out_row + rr] : (int64_t)(D.out_row + rr) * r;
    if (D.out_f32) {   // packed FP32 partial sums, FP32 output
        for (int c = cb; c < ce; ++c) {
            const float v = packed_sum(red + rr * rs + c, nrows * rs, G);
            float* dst = ws32 + orow + c0 + c;
            if (D.mode == SEG_STORE) *dst = v;
            else if (D.mode == SEG_ADD) *dst = __ldcg(dst) + v;
            else atomicAdd(dst, v);
        }
        return;
    }
    for (int c = cb; c < ce; ++c) {
        double s = 0.0;
        for (int g2 = 0; g2 < G; ++g2) s += red[(g2 * nrows + rr) * rs + c];
        double* dst = fin ? u2 + (int64_t)(c0 + c) * N + orow : ws + orow + c0 + c;
        if (D.mode == SEG_STORE || D.mode == SEG_FINAL) *dst = s;
        else if (D.mode == SEG_ADD) *dst = __ldcg(dst) + s;
        else atomicAdd(dst, s);   // SEG_ATOMIC; SEG_FINAL_ADD too (its value's only adder: the
                                  // same sum as a read-modify-write, without the load's latency)
    }
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) products of far-field chunks.
//
// A chunk of coupling or transfer blocks arrives as tensor tiles (see
// tc_offset).  The consumer warps split the operands into hi and lo parts in
// shared memory (TF32: hi = the nearest TF32 value, written back in place,
// lo = the nearest TF32 value of the remainder, so that |a - hi - lo| and
// |lo * lo| are below 2^-24 |a| and the tensor core's conversion is exact.
// BF16: the tiles already hold hi and lo), build the
// K-major B operand (the chunk's input vectors, N = r padded to the MMA's
// granularity, hi and lo), and one thread issues, per K step, the three
// products hi*hi + hi*lo + lo*hi into FP32 accumulators in tensor memory
// (M = 64 or 128 rows).  The accumulators live across the chunks of a
// segment; at its end the four warps that own the TMEM lane quarters read and
// add them (row i of an M = 128 tile is lane i; rows 16q..16q+15 of an M = 64 tile
// are lanes 32q..32q+15) and write the segment.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    // start address, K-direction core stride (LBO), row-group stride (SBO),
    // descriptor version 1 (bit 46), no swizzle
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint32_t mma_idesc(int type, int M, int N) {
    const uint32_t fmt = type == PIECE_TF32 ? 2u : 1u;   // TF32 (kind::tf32) or BF16 (kind::f16)
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_issue(int type, uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
    if (type == PIECE_TF32)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                     "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                     "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
                     : "memory");
}
// Nearest TF32 value of an FP32 number (ties away from zero): adding half a
// TF32 unit to the magnitude bits and clearing the 13 low mantissa bits.  The
// result is exactly representable in TF32, so the tensor core's own conversion
// leaves it unchanged.
__device__ __forceinline__ float tf32_rn(float v) {
    return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}
// Byte offset of B entry (n, kk) in a K-major operand of Np rows (K slow).
__device__ __forceinline__ int b_offset(int n, int kk, int Np, int es) {
    const int per = 16 / es;
    return (kk / per) * (Np / 8) * 128 + (n / 8) * 128 + (n % 8) * 16 + (kk % per) * es;
}

// Input columns a stage holds for r <= rt (see chunk_cols_for).
__host__ __device__ constexpr int xin_cols(int rt) { return rt > 8 ? 64 : kMaxChunkCols; }
// Input buffer of one stage: at most xin_cols(RT) FP64 rows of RT values
// plus the 16-byte rounding of every piece.
__host__ __device__ constexpr size_t xin_bytes(int rt) {
    return sizeof(double) * xin_cols(rt) * rt + 16 * H2_MAX_CHUNK_PIECES;
}
// The same for launches whose chunks all have FP32 inputs (the split form's
// far field): half the bytes, which leaves room for another stage.
__host__ __device__ constexpr size_t xin_bytes_f32(int rt) {
    return sizeof(float) * xin_cols(rt) * rt + 16 * H2_MAX_CHUNK_PIECES;
}

// Partial-sum buffers of the segment kernel: two, alternating between the
// reduction rounds of successive segments.
constexpr int kRedBuffers = 2;
// Right-hand sides per reduction round: all of them up to 8, else rounds of 4,
// which keeps the two buffers at 16 KB.  Rounds alternate between the
// buffers, so one consumer barrier per round suffices and nobody waits for
// the writers' global stores.
__host__ __device__ constexpr int red_rhs(int rt) { return rt <= 8 ? rt : 4; }

// Shared-memory layout of the segment kernel (dynamic part):
//   stages x stage_bytes             matrix chunks (bulk copies)
//   stages x a.xin_bytes             the chunks' input values (xin_bytes(RT), or
//                                    xin_bytes_f32(RT) where no chunk has FP64 inputs)
//   2 x kConsumers*red_rhs(RT)*8     partial sums of the row groups (two buffers)
//   tc_sets x (tc_alo_bytes + tc_b_bytes)   tensor-core operands (TF32 lo parts of A,
//                                    B with the rows of its vector parts)
//   stages x 2 + 5 mbarriers         full[], empty[], segment, operands-ready[2], products-done[2]
//
// Warp specialisation.  The producer warp (the last warp) walks this CTA's
// chunks: it waits until the consumers released the stage, issues the bulk
// copy of the chunk's matrices, copies the chunk's piece table into shared
// memory (one piece per lane), waits (dataflow form, first chunk of a
// segment, bounded) until the regions the segment reads are complete, copies
// the chunk's input values into the stage, publishes a descriptor and arrives
// on the stage's `full` barrier, which completes when the bulk copy has
// landed.  The 8 consumer warps wait on `full`, multiply, release the stage
// on `empty` and, at the end of a segment, add the row groups' partial sums
// (one mbarrier-based barrier among the consumers per reduction round); the
// writer warps write the segment and, in the dataflow form, each signals the
// segment's region with a release add.  No CTA-wide barrier is taken per
// chunk and no wait is unbounded.
// Registers: at r <= 16 (RT = 16, the split form's far-field launch) at most
// 96 (104 with the tensor-core path), so that this CTA and a near-field CTA
// at 64 registers share each SM sub-partition's 16 K registers even where
// three warps of each meet (3 x 32 x 104 + 3 x 32 x 64 <= 16384); otherwise
// as many as the 288 threads of one CTA per SM may take.
template <int RT, bool FLOW, bool TC>
__global__ void __maxnreg__(RT == 16 ? (TC ? 104 : 96) : 168) k_seg(const KArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = a.stages;
    const size_t xin_sz = (size_t)a.xin_bytes;
    constexpr int RR = red_rhs(RT);
    unsigned char* stage_base = smem;
    unsigned char* xbase = smem + (size_t)S * a.stage_bytes;
    double* red = reinterpret_cast<double*>(xbase + (size_t)S * xin_sz);
    // tensor-core operands after the partial sums;
    // operand set q: [lo parts of A][B: hi rows, lo rows] at tc_base + q * tc_set_bytes
    unsigned char* tc_base = reinterpret_cast<unsigned char*>(red + kRedBuffers * kConsumers * RR);
    const size_t tc_set_bytes = (size_t)a.tc_alo_bytes + (size_t)a.tc_b_bytes;
    const size_t red_span = (size_t)kRedBuffers * kConsumers * RR * sizeof(double);
    const size_t tc_span = (size_t)a.tc_sets * tc_set_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(red) + red_span + tc_span);
    uint64_t* empty = full + S;
    uint64_t* segbar = empty + S;
    uint64_t* cbar = segbar + 1;     // [2]: tensor operands of chunk n ready (barrier n & 1)
    uint64_t* mmabar = cbar + 2;     // [2]: tensor-core products of chunk n done (barrier n & 1)
    __shared__ StageDesc sd[kMaxStages];
    __shared__ SPiece spc[kMaxStages][H2_MAX_CHUNK_PIECES];
    __shared__ int abort_flag;
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 2);
            mbar_init(&empty[s], kConsumers);
        }
        mbar_init(segbar, kConsumers);
        mbar_init(&cbar[0], kConsumers - 32);   // the operand writers: consumer warps 1..7
        mbar_init(&cbar[1], kConsumers - 32);
        mbar_init(&mmabar[0], 1);
        mbar_init(&mmabar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (TC && tid < 32) {   // FP32 accumulators of up to 128 rows x Np right-hand sides
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(a.tc_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    volatile int* abortp = &abort_flag;
    int issued = 0;   // producer: chunks whose copy was issued

    if (tid >= kConsumers) {
        // ---------------- producer warp ----------------
        // The next segment (its descriptor and first 32 chunk descriptors,
        // one per lane) is fetched while the last chunk of the current one is
        // staged, so that the latencies overlap.
        const int lane = tid & 31;
        int k = 0;
        int nsg = -1;
        if (lane == 0) nsg = take_segment<FLOW>(a, k);
        nsg = __shfl_sync(~0u, nsg, 0);
        FlowSeg nF{};
        Chunk nmyc{};
        if (nsg >= 0) {
            nF = a.seg[nsg];
            if (lane < nF.s.nchunks) nmyc = a.chunk[nF.s.chunk0 + lane];
        }
        int sg = -1, ci = 0, base = 0;
        FlowSeg F{};
        Chunk myc{};     // chunk `base + lane` of the current segment
        for (int i = 0;; ++i) {
            const int st = i % S;
            if (i >= S) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_or_abort(&empty[st], (uint32_t)((i / S) - 1) & 1u, abortp);
                if (!__shfl_sync(~0u, ok, 0)) break;
            }
            if (sg < 0 || ci >= F.s.nchunks) {   // move to the prefetched segment
                sg = nsg;
                F = nF;
                myc = nmyc;
                ci = 0;
                base = 0;
            }
            if (sg < 0) {   // end marker: complete the phase without a copy
                if (lane == 0) {
                    sd[st].seg = -1;
                    mbar_arrive(&full[st]);
                    mbar_arrive(&full[st]);
                }
                break;
            }
            if (ci >= base + 32) {
                base += 32;
                if (base + lane < F.s.nchunks) myc = a.chunk[F.s.chunk0 + base + lane];
            }
            const int src_lane = ci - base;
            const long long csrc = __shfl_sync(~0u, (long long)myc.src, src_lane);
            const int cbytes = __shfl_sync(~0u, myc.bytes, src_lane);
            const int cpiece0 = __shfl_sync(~0u, myc.piece0, src_lane);
            const int cnp = __shfl_sync(~0u, myc.npieces, src_lane);
            const int cncols = __shfl_sync(~0u, myc.ncols, src_lane);
            const int cin0 = __shfl_sync(~0u, myc.in_row0, src_lane);
            const int ctype = __shfl_sync(~0u, myc.type0, src_lane);
            const bool f32 = ctype != PIECE_F64;   // FP32 inputs (FP32 workspace)
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load(stage_base + (size_t)st * a.stage_bytes, a.ctx[F.op].arena + csrc, (uint32_t)cbytes, &full[st]);
            }
            ++issued;
            const bool last = ci == F.s.nchunks - 1;
            if (last) {   // prefetch the next segment
                if (lane == 0) nsg = take_segment<FLOW>(a, k);
                nsg = __shfl_sync(~0u, nsg, 0);
                if (nsg >= 0) {
                    nF = a.seg[nsg];
                    if (lane < nF.s.nchunks) nmyc = a.chunk[nF.s.chunk0 + lane];
                }
            }
            // piece table of the chunk (one piece per lane), with the byte
            // offsets of the pieces' inputs in the stage's input buffer
            int in_total;
            if (cnp == 1) {
                in_total = input_bytes(cncols, a.ctx[F.op].r, f32);
                if (lane == 0) spc[st][0] = SPiece{0, cin0, cncols, 0};
            } else {
                Piece pc{};
                if (lane < cnp) pc = a.piece[cpiece0 + lane];
                const int mine = lane < cnp ? input_bytes(pc.ncols, a.ctx[F.op].r, f32) : 0;
                int xoff = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(~0u, xoff, o);
                    if (lane >= o) xoff += v;
                }
                in_total = __shfl_sync(~0u, xoff, 31);
                xoff -= mine;   // exclusive prefix
                if (lane < cnp) spc[st][lane] = SPiece{pc.smem_off, pc.in_row, pc.ncols, xoff};
            }
            // the chunk's inputs must fit the stage's input buffer (the host sizes it)
            bool ok = in_total <= a.xin_bytes;
            if (ok && FLOW && ci == 0 && lane == 0) ok = deps_wait(a, F, abortp);
            if (!__shfl_sync(~0u, ok, 0)) {
                if (lane == 0) {
                    atomicExch(a.err, 1);
                    abort_flag = 1;
                    sd[st].seg = -1;
                    mbar_arrive(&full[st]);
                }
                break;
            }
            if (lane == 0)
                asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[st])),
                             "r"(in_total)
                             : "memory");
            __syncwarp();
            issue_inputs(a.ctx[F.op], spc[st], cnp, f32, xbase + (size_t)st * xin_sz, &full[st], lane);
            if (lane == 0) {
                StageDesc D;
                D.seg = sg;
                D.last = last;
                D.npieces = cnp;
                D.f32 = f32;
                D.out_row = F.s.out_row;
                D.nrows = F.s.nrows;
                D.mode = F.s.mode;
                D.out_f32 = F.s.out_f32;
                D.ptype = ctype;
                D.cbytes = cbytes;
                D.op = F.op;
                D.signal = F.signal;
                sd[st] = D;
                mbar_arrive(&full[st]);
            }
            ++ci;
        }
    } else {
        // ---------------- consumer warps ----------------
        double acc[RT];   // FP64 sums, or packed compensated FP32 sums (segments with FP32 output)
        double acc1 = 0.0;   // second FP64 chain at RT = 1
#pragma unroll
        for (int c = 0; c < RT; ++c) acc[c] = 0.0;
        uint32_t segphase = 0;
        int tcn = 0;            // tensor-core chunks so far
        int segk = 0;           // K steps of the current tensor-core segment issued so far
        int pend_st = -1;       // stage of the last tensor-core chunk, released once its products are done
        int pend_n = 0;
        auto release_pending = [&]() -> bool {
            if (!TC || pend_st < 0) return true;
            if (!mbar_wait_or_abort(&mmabar[pend_n & 1], (uint32_t)(pend_n >> 1) & 1u, abortp)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mbar_arrive(&empty[pend_st]);
            pend_st = -1;
            return true;
        };
        for (int i = 0;; ++i) {
            const int st = i % S;
            if (!mbar_wait_or_abort(&full[st], (uint32_t)(i / S) & 1u, abortp)) {
                atomicExch(a.err, 1);
                abort_flag = 1;
                break;
            }
            const StageDesc D = sd[st];
            if (D.seg < 0) break;
            const OpCtx& C = a.ctx[D.op];
            const int r = C.r;
            if (TC && piece_tc(D.ptype) && !a.tc_cuda) {
                // ---------- tensor-core chunk ----------
                unsigned char* stg = stage_base + (size_t)st * a.stage_bytes;
                const unsigned char* xin = xbase + (size_t)st * xin_sz;
                const int type = D.ptype;
                const int Mp = tc_rows(D.nrows);
                const int Np = Mp == 64 ? (r + 7) / 8 * 8 : (r + 15) / 16 * 16;
                const int ks = tc_kstep(type);
                const int bes = type == PIECE_TF32 ? 4 : 2;
                // vector parts: TF32 hi, lo; BF16 hi, mid, lo (exact for the FP32 vector)
                const int ph = type == PIECE_TF32 ? 2 : 3;
                // one operand set: wait until the previous chunk's products are done
                if (a.tc_sets == 1 && !release_pending()) {
                    atomicExch(a.err, 1);
                    abort_flag = 1;
                    break;
                }
                unsigned char* set = tc_base + (size_t)(tcn % a.tc_sets) * tc_set_bytes;
                unsigned char* t_alo = set;
                unsigned char* t_b = set + a.tc_alo_bytes;   // B: ph x Np rows, part by part
                const int Nt = ph * Np;
                // operands: written by consumer warps 1..7 while warp 0 issues the
                // previous chunk's products
                const int wt = tid - 32, nwt = kConsumers - 32;
                if (type == PIECE_TF32 && wt >= 0) {   // A = hi (in place) + lo, both nearest TF32 values
                    float4* A4 = reinterpret_cast<float4*>(stg);
                    float4* L4 = reinterpret_cast<float4*>(t_alo);
                    for (int q = wt; q < D.cbytes / 16; q += nwt) {
                        const float4 v = A4[q];
                        const float4 h = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
                        A4[q] = h;
                        L4[q] = make_float4(tf32_rn(v.x - h.x), tf32_rn(v.y - h.y), tf32_rn(v.z - h.z),
                                            tf32_rn(v.w - h.w));
                    }
                }
                // B operand: part p of right-hand side n is row p * Np + n, K = the
                // pieces' input rows (each piece padded to whole K steps with zeros).
                // Rows r..Np-1 of each part are not written: they only reach
                // accumulator columns that are never read.  A work unit is one 16-byte
                // core row: right-hand side n, `per` consecutive K rows (8 BF16 or 4
                // TF32 values), written with one vector store per part.  TF32: hi =
                // RN_tf32(x), lo = RN_tf32(x - hi).  BF16: hi = bf16(x), mid =
                // bf16(x - hi), lo = bf16(x - hi - mid); both differences are exact in
                // FP32 and the last one has at most 8 significant bits, so hi + mid +
                // lo = x exactly.
                if (wt >= 0) {
                    const int per = 16 / bes;
                    const int nb = r;
                    int kb = 0;
                    for (int p = 0; p < D.npieces; ++p) {
                        const SPiece P = spc[st][p];
                        const int kp = (P.ncols + ks - 1) / ks * ks;
                        const float* xp = reinterpret_cast<const float*>(xin + P.xoff);
                        const int units = (kp / per) * nb;
                        for (int u = wt; u < units; u += nwt) {
                            const int kg = u / nb, n = u - kg * nb;   // K group, right-hand side
                            const int j0 = kg * per;
                            const int off0 = b_offset(n, kb + j0, Nt, bes);
                            const int off1 = b_offset(Np + n, kb + j0, Nt, bes);
                            if (type == PIECE_TF32) {
                                float h[4], l[4];
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const float x = (j0 + e < P.ncols && n < r) ? xp[(j0 + e) * r + n] : 0.0f;
                                    h[e] = tf32_rn(x);
                                    l[e] = tf32_rn(x - h[e]);
                                }
                                *reinterpret_cast<float4*>(t_b + off0) = make_float4(h[0], h[1], h[2], h[3]);
                                *reinterpret_cast<float4*>(t_b + off1) = make_float4(l[0], l[1], l[2], l[3]);
                            } else {
                                const int off2 = b_offset(2 * Np + n, kb + j0, Nt, bes);
                                __align__(16) __nv_bfloat16 h[8], mi[8], l[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) {
                                    const float x = (j0 + e < P.ncols && n < r) ? xp[(j0 + e) * r + n] : 0.0f;
                                    h[e] = __float2bfloat16_rn(x);
                                    const float d1 = x - __bfloat162float(h[e]);
                                    mi[e] = __float2bfloat16_rn(d1);
                                    l[e] = __float2bfloat16_rn(d1 - __bfloat162float(mi[e]));
                                }
                                *reinterpret_cast<uint4*>(t_b + off0) = *reinterpret_cast<const uint4*>(h);
                                *reinterpret_cast<uint4*>(t_b + off1) = *reinterpret_cast<const uint4*>(mi);
                                *reinterpret_cast<uint4*>(t_b + off2) = *reinterpret_cast<const uint4*>(l);
                            }
                        }
                        kb += kp;
                    }
                }
                if (wt >= 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(&cbar[tcn & 1]);
                }
                // K steps of this chunk (every consumer thread tracks the segment's count)
                int csteps = 0;
                for (int p = 0; p < D.npieces; ++p) csteps += (spc[st][p].ncols + ks - 1) / ks;
                // accumulator columns in tensor memory: nacc A_hi accumulators of whi
                // columns, then ncorr A_lo accumulators of wlo columns
                const uint32_t whi = (uint32_t)(a.tc_parts * a.tc_np), wlo = (uint32_t)((a.tc_parts - 1) * a.tc_np);
                if (tid == 0) {
                    // Per K step two products: A_hi x B (N = ph Np: A_hi times every
                    // part of the vector) into accumulator g % nacc, and A_lo x B's
                    // first ph - 1 parts (N = (ph - 1) Np: A_lo times all but the
                    // vector's lowest part) into correction accumulator g % ncorr.
                    // Products into one accumulator wait for each other, into
                    // different ones overlap.
                    bool ok = mbar_wait_or_abort(&cbar[tcn & 1], (uint32_t)(tcn >> 1) & 1u, abortp);
                    if (!ok) {
                        atomicExch(a.err, 1);
                        abort_flag = 1;
                    } else {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t idesc_h = mma_idesc(type, Mp, Nt), idesc_l = mma_idesc(type, Mp, Nt - Np);
                        const uint32_t lboA = 16u * Mp, lboB = (uint32_t)(Nt / 8) * 128u;
                        const int bper = 16 / bes;
                        const int nacc = a.tc_nacc, ncorr = a.tc_ncorr;
                        const uint32_t tcorr0 = tmem_base + (uint32_t)nacc * whi;
                        // descriptors advance by adding (byte offset >> 4) to their
                        // 14-bit start-address field (shared memory < 256 KB: no carry)
                        const uint64_t dA0 = smem_desc(smem_addr(stg), lboA, 128);
                        const uint64_t dL0 = type == PIECE_TF32 ? smem_desc(smem_addr(t_alo), lboA, 128)
                                                                : dA0 + (uint64_t)((32u * Mp) >> 4);
                        const uint64_t dB = smem_desc(smem_addr(t_b), lboB, 128);
                        const uint64_t a_step = (uint64_t)((ks * Mp * 4) >> 4);        // one K slab of A
                        const uint64_t b_step = (uint64_t)(((ks / bper) * lboB) >> 4);  // one K step of B
                        int gstep = segk;
                        int accn = segk % nacc, corn = segk % ncorr;
                        uint64_t bo = 0;
                        for (int p = 0; p < D.npieces; ++p) {
                            const SPiece P = spc[st][p];
                            const int nst = (P.ncols + ks - 1) / ks;
                            uint64_t ao = (uint64_t)(P.smem_off >> 4);
                            for (int k2 = 0; k2 < nst; ++k2, ++gstep, ao += a_step, bo += b_step) {
                                mma_issue(type, tmem_base + (uint32_t)accn * whi, dA0 + ao, dB + bo, idesc_h,
                                          gstep >= nacc ? 1u : 0u);
                                mma_issue(type, tcorr0 + (uint32_t)corn * wlo, dL0 + ao, dB + bo, idesc_l,
                                          gstep >= ncorr ? 1u : 0u);
                                if (++accn == nacc) accn = 0;
                                if (++corn == ncorr) corn = 0;
                            }
                        }
                    }
                    // committed also after an abort, so that the bounded waits on it end
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_addr(&mmabar[tcn & 1]))
                                 : "memory");
                }
                if (*abortp) break;
                segk += csteps;
                // accumulators written: A_hi ones, then correction ones
                const int nused = segk < a.tc_nacc ? segk : a.tc_nacc;
                const int ncused = segk < a.tc_ncorr ? segk : a.tc_ncorr;
                // the previous chunk's products are done by now in the common case
                if (!release_pending()) {
                    atomicExch(a.err, 1);
                    abort_flag = 1;
                    break;
                }
                pend_st = st;
                pend_n = tcn++;
                if (D.last) {
                    if (!release_pending()) {
                        atomicExch(a.err, 1);
                        abort_flag = 1;
                        break;
                    }
                    if (tid < 128) {   // the four lane-quarter warps read and add the accumulators
                        const int w = tid >> 5, lane = tid & 31;
                        const int row = Mp == 128 ? tid : (lane < 16 ? 16 * w + lane : -1);
                        const uint32_t tlane = tmem_base + ((uint32_t)(32 * w) << 16);
                        float* dst = C.ws32 + (int64_t)(D.out_row + (row < 0 ? 0 : row)) * r;
                        // column groups to add: every part of each A_hi accumulator, then
                        // the first ph - 1 parts of each correction accumulator
                        const int nhi = ph * nused, ntot = nhi + (ph - 1) * ncused;
                        for (int c0 = 0; c0 < Np; c0 += 8) {   // 8 right-hand sides at a time
                            float sum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                            for (int j = 0; j < ntot; ++j) {
                                const uint32_t col =
                                    j < nhi ? (uint32_t)(j / ph) * whi + (uint32_t)((j % ph) * Np + c0)
                                            : (uint32_t)a.tc_nacc * whi + (uint32_t)((j - nhi) / (ph - 1)) * wlo +
                                                  (uint32_t)(((j - nhi) % (ph - 1)) * Np + c0);
                                uint32_t v[8];
                                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]),
                                               "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                                             : "r"(tlane + col));
                                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                                for (int c = 0; c < 8; ++c) sum[c] += __uint_as_float(v[c]);
                            }
                            if (row >= 0 && row < D.nrows) {
#pragma unroll
                                for (int c = 0; c < 8; ++c) {
                                    if (c0 + c >= r) break;
                                    float* d = dst + c0 + c;
                                    if (D.mode == SEG_STORE) *d = sum[c];
                                    else if (D.mode == SEG_ADD) *d = __ldcg(d) + sum[c];
                                    else atomicAdd(d, sum[c]);
                                }
                            }
                        }
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        if (FLOW && D.signal >= 0) {   // one unit per 16-row group of the segment it wrote
                            const int ng = Mp == 128 ? (32 * w < D.nrows) + (32 * w + 16 < D.nrows) : (16 * w < D.nrows);
                            __syncwarp();
                            if (lane == 0 && ng > 0) signal_region(a.cnt + D.signal, ng);
                        }
                    }
                    segk = 0;
                }
                continue;
            }
            // a CUDA-core chunk: the tensor core must be done with the operand
            // sets (the partial sums may share their memory) and the stage
            if (!release_pending()) {
                atomicExch(a.err, 1);
                abort_flag = 1;
                break;
            }
            const int nrows = D.nrows;
            const int G = kConsumers / nrows;
            const int row = tid % nrows, g = tid / nrows;
            if (g < G) {
                bool done = false;
                if constexpr (!TC) {   // evaluated coupling blocks (FP32 operators)
                    if (D.ptype == PIECE_NODES) {
                        const int t = (int)((D.out_row - C.row_yhat) / C.kp);
                        consume_nodes<RT>(stage_base + (size_t)st * a.stage_bytes, spc[st], D.npieces,
                                          xbase + (size_t)st * xin_sz, r, C.nodes[(int64_t)t * C.kp + row], g, G,
                                          acc);
                        done = true;
                    }
                }
                if constexpr (!TC && RT <= kTcCudaMaxRT) {   // tensor tiles on the CUDA cores (a.tc_cuda)
                    if (!done && piece_tc(D.ptype)) {
                        consume_tc_tiles<RT>(stage_base + (size_t)st * a.stage_bytes, spc[st], D.npieces, D.ptype,
                                             xbase + (size_t)st * xin_sz, r, nrows, row, g, G, acc);
                        done = true;
                    }
                }
                if (!done)
                    consume_chunk<RT>(stage_base + (size_t)st * a.stage_bytes, spc[st], D.npieces, D.f32 != 0,
                                      xbase + (size_t)st * xin_sz, r, nrows, row, g, G, D.out_f32 != 0, acc, acc1);
            }
            mbar_arrive(&empty[st]);
            if (D.last) {
                // partial sums of the row groups, RR right-hand sides per round
                bool ok = true;
                const bool writer = (tid >> 5) < writer_warps(nrows);
#pragma unroll
                for (int q = 0; q < RT / RR; ++q) {
                    if (q * RR >= r) break;
                    double* rb = red + (size_t)(segphase % kRedBuffers) * kConsumers * RR;
                    if (g < G) {
#pragma unroll
                        for (int c = 0; c < RR; ++c) rb[tid * RR + c] = acc[q * RR + c];   // packed sums as they are
                        if (RT == 1 && !D.out_f32) rb[tid] = acc[0] + acc1;
                    }
                    mbar_arrive(segbar);
                    if (!(ok = mbar_wait_or_abort(segbar, segphase++ & 1u, abortp))) break;
                    if (writer) {
                        const int cn = r - q * RR < RR ? r - q * RR : RR;
                        write_segment(D, rb, RR, q * RR, cn, r, G, C.ws, C.ws32, C.u2, C.perm, C.N);
                    }
                }
                if (!ok) {
                    atomicExch(a.err, 1);
                    abort_flag = 1;
                    break;
                }
#pragma unroll
                for (int c = 0; c < RT; ++c) acc[c] = 0.0;
                acc1 = 0.0;
                if (FLOW && writer && D.signal >= 0) {
                    __syncwarp();
                    if ((tid & 31) == 0) signal_region(a.cnt + D.signal);
                }
            }
        }
        // the tensor core finishes before its memory is released (bounded)
        (void)release_pending();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // after an abort, let the producer's copies still in flight land (bounded)
    if (tid == kConsumers && abort_flag) {
        for (int j = issued > S ? issued - S : 0; j < issued; ++j)
            (void)mbar_wait(&full[j % S], (uint32_t)(j / S) & 1u);
    }
    if (TC && tid < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(a.tc_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Near field of the split form (r > 8, reduced-precision operators): the FP64
// near blocks N_ts of every leaf t (Section "H2-Matrix Compression": the
// inadmissible blocks, exact Lindholm entries, Psi on the diagonal of N_tt)
// applied to all r right-hand sides and stored in `u2n` (r x N, mesh order).
// It runs beside the far-field launch, which then has no FP64 work: the FP64
// pipe and the tensor / FP32 pipes of an SM work at the same time.  One
// producer warp stages each chunk as in k_seg (bulk copies of the matrices
// and of their input rows); the eight consumer warps take the nrows x r
// outputs of a segment as work items (row, right-hand side) dealt round-robin
// to their 256 threads, every item over every column, so that no partial sums
// meet across threads and the four SM sub-partitions get equal shares of the
// FP64 work (two warps each, so that one's dependency waits are the other's
// issue slots).  The CTAs take work units from an atomic ticket, longest
// first: a segment, or a run of its chunks where a few SMs would otherwise
// finish the largest leaves alone; a unit's sums are added to the cleared
// u2n (a value receives one addition per unit of its leaf).  No unit waits
// for another.  The paired form (PAIR, h2_near_field H2_NEAR_F32PAIR) stages
// the paired copy of the blocks and the paired inputs (8 bytes per value as
// in FP64) and gives each thread one output row and four consecutive
// right-hand sides instead, so that one entry load serves four products.
// ---------------------------------------------------------------------------
// Consumer threads of the near-field kernel: twelve warps for the FP64 items
// (three per SM sub-partition, so that two of them can wait on their operand
// loads while the third keeps the FP64 pipe busy), eight for the paired form.
template <bool PAIR>
__host__ __device__ constexpr int near_cons() {
    return PAIR ? 256 : 384;
}

// One term a*x of a paired near-field sum hi + lo (h2_near_field
// H2_NEAR_F32PAIR; a, x = (hi, lo) FP32 pairs): the product of the high words
// is split exactly into its rounded value p and error e (an FMA gives e,
// Dekker 1971); p enters hi through TwoSum (Knuth), whose error, e and the
// cross terms a.hi*x.lo + a.lo*x.hi go to lo (a.lo*x.lo, below 2^-48 of the
// term, is left out).  p is taken with __fmul_rn so that the compiler cannot
// contract it into the sum.
__device__ __forceinline__ void pair_fma(float2 a, float2 x, float& hi, float& lo) {
    const float p = __fmul_rn(a.x, x.x);
    const float e = fmaf(a.x, x.x, -p);
    float s, t;
    two_sum(hi, p, s, t);
    hi = s;
    lo = fmaf(a.x, x.y, lo);
    lo = fmaf(a.y, x.x, lo);
    lo += e + t;
}

struct NArgs {
    const FlowSeg* seg;     // the near pass's segments (leaves, <= 64 rows)
    const Chunk* chunk;
    const Piece* piece;
    const int4* units;      // work units: segment, first chunk in it, chunks
    int nunits;
    const unsigned char* arena;   // chunk c's bytes at arena + (c.src - src_base)
    int64_t src_base;
    const unsigned char* xsrc;    // input rows in tree order, 8 bytes per value:
                                  // FP64, or an FP32 pair (hi, lo) when PAIR
    double* u2n;            // r x N
    const int32_t* perm;
    int64_t N;
    int r;
    int stages, stage_bytes;
    int32_t* ticket;        // cleared by the gather
    int32_t* err;
};

struct NStage {
    int32_t seg, last, npieces, out_row, nrows;
};

// NJ (row, right-hand side) items of one thread over the columns of a staged
// FP64 near block (column-major, nrows rows; inputs r values per column).
// NJ is the same for every lane of a warp, so a warp whose item slots lie
// beyond the unit's items issues no FP64 instruction for them: an FMA with
// its lanes predicated off would still hold the FP64 pipe.
// Item j of a thread is packed as row | (right-hand side << 8) (rows <= 64,
// right-hand sides <= 16).  The operands of column col + 1 are loaded before
// the FMAs of column col issue: the FP64 pipe takes one warp FMA per 64
// cycles per SM sub-partition, so a warp waits at its FMAs, and loads issued
// behind them would leave the pipe idle for their latency whenever both of
// the sub-partition's consumer warps reach a new column together.
template <int NJ, int JM>
__device__ __forceinline__ void near_item_cols(const double* __restrict__ A, const double* __restrict__ x, int nrows,
                                               int r, int ncols, const int (&item)[JM], double (&acc)[JM]) {
    if (ncols <= 0) return;
    int ao[NJ], xo[NJ];
    double av[NJ], xv[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        ao[j] = item[j] & 0xFF;
        xo[j] = item[j] >> 8;
        av[j] = A[ao[j]];
        xv[j] = x[xo[j]];
    }
#pragma unroll 1
    for (int col = 1; col < ncols; ++col) {
        const double* Ac = A + col * nrows;
        const double* xc = x + col * r;
        double an[NJ], xn[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            an[j] = Ac[ao[j]];
            xn[j] = xc[xo[j]];
        }
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            acc[j] = fma(av[j], xv[j], acc[j]);
            av[j] = an[j];
            xv[j] = xn[j];
        }
    }
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = fma(av[j], xv[j], acc[j]);
}

// At most 48 registers per thread (the paired form: 40): one CTA of this
// kernel and one of the far-field launch at r <= 16 (288 threads x at most 104
// registers) share each SM sub-partition's 16 K registers even where four
// warps of this one meet three of the other (4 x 32 x 48 + 3 x 32 x 104 <=
// 16384).
template <int RT, bool PAIR>
__global__ void __maxnreg__(PAIR ? 40 : 48) k_near_items(const NArgs a) {
    constexpr int NC = near_cons<PAIR>();
    // items per thread: 64 rows x RT over the NC threads (paired: four
    // right-hand sides of one row)
    constexpr int JM = PAIR ? RT / 4 : (64 * RT + NC - 1) / NC;
    static_assert(!PAIR || JM >= 4, "paired form: four right-hand sides per thread");
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = a.stages;
    constexpr size_t kXin = xin_bytes(RT);
    unsigned char* stage_base = smem;
    unsigned char* xbase = smem + (size_t)S * a.stage_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(xbase + (size_t)S * kXin);
    uint64_t* empty = full + S;
    __shared__ NStage sd[kMaxStages];
    __shared__ SPiece spc[kMaxStages][H2_MAX_CHUNK_PIECES];
    __shared__ int abort_flag;
    const int tid = threadIdx.x;
    if (tid == 0) {
        abort_flag = 0;
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 2);
            mbar_init(&empty[q], NC);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abortp = &abort_flag;
    int issued = 0;
    const int r = a.r;
    if (tid >= NC) {
        // ---------------- producer warp ----------------
        const int lane = tid & 31;
        int i = 0;
        bool ok = true;
        while (ok) {
            int un = 0;
            if (lane == 0) un = atomicAdd(a.ticket, 1);
            un = __shfl_sync(~0u, un, 0);
            const bool end = un >= a.nunits;
            const int4 U = end ? make_int4(0, 0, 1, 0) : a.units[un];
            const Segment F = end ? Segment{} : a.seg[U.x].s;
            for (int ci = 0; ci < U.z; ++ci, ++i) {
                const int st = i % S;
                if (i >= S) {
                    bool w = true;
                    if (lane == 0) w = mbar_wait_or_abort(&empty[st], (uint32_t)((i / S) - 1) & 1u, abortp);
                    if (!__shfl_sync(~0u, w, 0)) {
                        if (lane == 0) {
                            atomicExch(a.err, 1);
                            abort_flag = 1;
                        }
                        ok = false;
                        break;
                    }
                }
                if (end) {   // end marker: complete the phase without a copy
                    if (lane == 0) {
                        sd[st].seg = -1;
                        mbar_arrive(&full[st]);
                        mbar_arrive(&full[st]);
                    }
                    ok = false;
                    break;
                }
                const Chunk ch = a.chunk[F.chunk0 + U.y + ci];
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tma_load(stage_base + (size_t)st * a.stage_bytes, a.arena + (ch.src - a.src_base),
                             (uint32_t)ch.bytes, &full[st]);
                }
                ++issued;
                Piece pc{};
                if (lane < ch.npieces) pc = a.piece[ch.piece0 + lane];
                const int mine = lane < ch.npieces ? input_bytes(pc.ncols, r, false) : 0;
                int xoff = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(~0u, xoff, o);
                    if (lane >= o) xoff += v;
                }
                const int in_total = __shfl_sync(~0u, xoff, 31);
                xoff -= mine;
                if (lane < ch.npieces) spc[st][lane] = SPiece{pc.smem_off, pc.in_row, pc.ncols, xoff};
                if (lane == 0)
                    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&full[st])),
                                 "r"(in_total)
                                 : "memory");
                __syncwarp();
                if (lane < ch.npieces) {
                    asm volatile("fence.proxy.async.global;" ::: "memory");
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_addr(xbase + (size_t)st * kXin + xoff)),
                        "l"(a.xsrc + (int64_t)pc.in_row * r * 8), "r"(mine), "r"(smem_addr(&full[st]))
                        : "memory");
                }
                if (lane == 0) {
                    sd[st] = NStage{un, ci == U.z - 1, ch.npieces, F.out_row, F.nrows};
                    mbar_arrive(&full[st]);
                }
            }
        }
    } else {
        // ---------------- consumer warps ----------------
        double acc[JM];
        float hi[JM], lo[JM];   // PAIR: each item's running sum hi + lo
#pragma unroll
        for (int j = 0; j < JM; ++j) {
            acc[j] = 0.0;
            hi[j] = 0.0f;
            lo[j] = 0.0f;
        }
        int cur = -1, nitems = 0, nrows = 1;
        int item[JM];             // item j of this thread: output row | (right-hand side << 8)
        int nj = 0;               // item slots of this warp that hold items (the same on every lane)
        // PAIR: one output row and up to four consecutive right-hand sides per
        // thread (64 rows x 16 right-hand sides fill the 256 threads), so that
        // one entry load serves four products
        int prow = 0, prhs0 = 0, pcnt = 0;
        for (int i = 0;; ++i) {
            const int st = i % S;
            if (!mbar_wait_or_abort(&full[st], (uint32_t)(i / S) & 1u, abortp)) {
                atomicExch(a.err, 1);
                abort_flag = 1;
                break;
            }
            const NStage D = sd[st];
            if (D.seg < 0) break;
            if (D.seg != cur) {   // items of a new work unit
                cur = D.seg;
                nrows = D.nrows;
                nitems = nrows * r;
                if constexpr (PAIR) {
                    prow = tid % nrows;
                    prhs0 = tid / nrows * 4;
                    pcnt = tid < nrows * ((r + 3) / 4) ? min(4, r - prhs0) : 0;
                } else {
                    // slot j of lane l of warp w: item 32 w + l + 256 j; slots past the
                    // items point at item 0 (their sums are never written)
                    nj = 0;
#pragma unroll
                    for (int j = 0; j < JM; ++j) {
                        const int it = tid + NC * j;
                        item[j] = it < nitems ? (it % nrows) | ((it / nrows) << 8) : 0;
                        if ((tid & ~31) + NC * j < nitems) nj = j + 1;
                    }
                }
            }
            const unsigned char* stg = stage_base + (size_t)st * a.stage_bytes;
            const unsigned char* xin = xbase + (size_t)st * kXin;
            for (int p = 0; p < D.npieces; ++p) {
                const SPiece P = spc[st][p];
                if constexpr (PAIR) {
                    const float2* A = reinterpret_cast<const float2*>(stg + P.smem_off) + prow;
                    const float2* x = reinterpret_cast<const float2*>(xin + P.xoff) + prhs0;
                    if (pcnt == 4) {
#pragma unroll 2
                        for (int col = 0; col < P.ncols; ++col) {
                            const float2 av = A[col * nrows];
                            const float2* xc = x + col * r;
                            pair_fma(av, xc[0], hi[0], lo[0]);
                            pair_fma(av, xc[1], hi[1], lo[1]);
                            pair_fma(av, xc[2], hi[2], lo[2]);
                            pair_fma(av, xc[3], hi[3], lo[3]);
                        }
                    } else if (pcnt > 0) {
                        for (int col = 0; col < P.ncols; ++col) {
                            const float2 av = A[col * nrows];
                            const float2* xc = x + col * r;
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (j < pcnt) pair_fma(av, xc[j], hi[j], lo[j]);
                        }
                    }
                } else {
                    const double* A = reinterpret_cast<const double*>(stg + P.smem_off);
                    const double* x = reinterpret_cast<const double*>(xin + P.xoff);
                    static_assert(JM == 3, "the FP64 item form is instantiated for 16 right-hand sides");
                    switch (nj) {   // warp-uniform
                        case 3: near_item_cols<3>(A, x, nrows, r, P.ncols, item, acc); break;
                        case 2: near_item_cols<2>(A, x, nrows, r, P.ncols, item, acc); break;
                        case 1: near_item_cols<1>(A, x, nrows, r, P.ncols, item, acc); break;
                        default: break;
                    }
                }
            }
            mbar_arrive(&empty[st]);
            if (D.last) {
#pragma unroll
                for (int j = 0; j < JM; ++j) {
                    if constexpr (PAIR) {
                        if (j < pcnt)
                            atomicAdd(a.u2n + (int64_t)(prhs0 + j) * a.N + a.perm[D.out_row + prow],
                                      (double)hi[j] + (double)lo[j]);
                    } else {
                        if (tid + NC * j < nitems)
                            atomicAdd(a.u2n + (int64_t)(item[j] >> 8) * a.N + a.perm[D.out_row + (item[j] & 0xFF)],
                                      acc[j]);
                    }
                    acc[j] = 0.0;
                    hi[j] = 0.0f;
                    lo[j] = 0.0f;
                }
            }
        }
    }
    __syncthreads();
    // after an abort, let the producer's copies still in flight land (bounded)
    if (tid == NC && abort_flag) {
        for (int j = issued > S ? issued - S : 0; j < issued; ++j)
            (void)mbar_wait(&full[j % S], (uint32_t)(j / S) & 1u);
    }
}

// u2 += u2n over n values (the split form's near field).
__global__ void k_add(double* __restrict__ u2, const double* __restrict__ u2n, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u2[i] += u2n[i];
}

// Gathers the input into the workspace's input rows (leaf by leaf in tree
// order, padding rows zero) in FP64 and, for FP32 operators, in FP32 and, for
// a paired near field, as FP32 pairs hi = fp32(v), lo = fp32(v - hi); clears
// the y-hat rows that are accumulated atomically (in the workspace of the
// far field); clears `nclear` ints (the flow kernel's counters).
__global__ void k_prologue(const double* __restrict__ u1, double* __restrict__ ws, float* __restrict__ ws32,
                           float2* __restrict__ wsp, const int32_t* __restrict__ gsrc, int64_t nrows_in, int64_t N, int r,
                           const int32_t* __restrict__ zero_rows, int nzero, int kp, int32_t* __restrict__ clear,
                           int nclear) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = nrows_in * r;
    for (int64_t idx = i0; idx < tot; idx += stride) {
        const int64_t q = idx / r, c = idx - q * r;
        const int32_t src = gsrc[q];
        const double v = src >= 0 ? u1[c * N + src] : 0.0;
        ws[idx] = v;
        if (ws32) ws32[idx] = (float)v;
        if (wsp) {
            const float h = __double2float_rn(v);
            wsp[idx] = make_float2(h, __double2float_rn(v - (double)h));
        }
    }
    const int64_t per = (int64_t)kp * r;
    const int64_t totz = (int64_t)nzero * per;
    for (int64_t idx = i0; idx < totz; idx += stride) {
        const int64_t z = idx / per, j = idx - z * per;
        if (ws32) ws32[(int64_t)zero_rows[z] * r + j] = 0.0f;
        else ws[(int64_t)zero_rows[z] * r + j] = 0.0;
    }
    for (int64_t idx = i0; idx < nclear; idx += stride) clear[idx] = 0;
}

int stages_for(int rt, int stage_bytes, int alo, int b);
static int tc_alo_bytes(const h2_handle* op);
static int tc_b_bytes(const h2_handle* op, int rt);
// The operator's stage count: the autotuner's choice, else the default.
static int op_stages(const h2_handle* op, int rt) {
    return op && op->tune_stages > 0 ? op->tune_stages
                                     : stages_for(rt, op->stage_bytes, tc_alo_bytes(op), tc_b_bytes(op, rt));
}

int rt_for(int r) {
    int rt = 1;
    while (rt < r) rt *= 2;
    return rt;
}

// Allows `smem` bytes of dynamic shared memory and asks for the largest
// shared-memory carveout, so that as many CTAs as fit are resident per SM.
// One record per kernel for every path that launches or sizes it: a path with
// a record of its own could lower the kernel's limit below what another
// path's record still assumes, and that path's next launch would fail.
template <class F>
cudaError_t set_smem(F* kernel, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void*, size_t> configured;
    std::lock_guard<std::mutex> lock(mu);
    size_t& c = configured[reinterpret_cast<const void*>(kernel)];
    if (c >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) c = smem;
    return e;
}

// Resident CTAs per SM of a kernel at this shared-memory size (cached).
template <class F>
int ctas_per_sm(F* kernel, size_t smem, int& cached, size_t& cached_smem) {
    if (cached > 0 && cached_smem == smem) return cached;
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kBlock, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    cached = n;
    cached_smem = smem;
    return n;
}

// Launches `nsm` x (resident CTAs per SM) CTAs (at most one per segment);
// *launched receives the grid size.
template <int RT, bool FLOW, bool TC>
cudaError_t launch_seg_rt(const KArgs& a, int nsm, size_t smem, cudaStream_t s, int* launched, int cap) {
    static size_t occ_smem = 0;
    static int occ = 0;
    cudaError_t e = set_smem(k_seg<RT, FLOW, TC>, smem);
    if (e != cudaSuccess) return e;
    int per_sm = ctas_per_sm(k_seg<RT, FLOW, TC>, smem, occ, occ_smem);
    if (cap > 0 && cap < per_sm) per_sm = cap;   // the autotuner's CTA count
    const int g = std::max(1, std::min(a.nseg, nsm * per_sm));
    if (launched) *launched = g;
    KArgs b = a;
    if (TC) {
        // TMEM columns per CTA: a power of 2 such that the resident CTAs of an SM
        // never ask for more than its 512 columns (an allocation never waits);
        // about half of them take the A_hi accumulators (all `parts` vector parts
        // of np columns each), the rest the A_lo corrections (parts - 1 of them)
        int cols = 512;
        while (cols * per_sm > 512 && cols > 32) cols >>= 1;
        const int np = (a.r + 15) / 16 * 16;
        const int parts = a.tc_parts >= 2 ? a.tc_parts : 2;
        const int whi = parts * np, wlo = (parts - 1) * np;
        if (cols < whi + wlo) return cudaErrorInvalidConfiguration;
        b.tc_parts = parts;
        b.tc_cols = cols;
        b.tc_np = np;
        b.tc_nacc = std::max(1, std::min(8, (cols / 2) / whi));
        b.tc_ncorr = std::max(1, std::min(8, (cols - whi * b.tc_nacc) / wlo));
    }
    k_seg<RT, FLOW, TC><<<g, kBlock, smem, s>>>(b);
    return cudaGetLastError();
}

template <int RT, bool TC>
int seg_occupancy(size_t smem) {
    if (set_smem(k_seg<RT, true, TC>, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_seg<RT, true, TC>, kBlock, smem) != cudaSuccess ||
        n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

template <bool FLOW, bool TC>
cudaError_t launch_seg_tc(const KArgs& a, int rt, int nsm, size_t smem, cudaStream_t s, int* launched, int cap) {
    switch (rt) {
        case 1: return launch_seg_rt<1, FLOW, TC>(a, nsm, smem, s, launched, cap);
        case 2: return launch_seg_rt<2, FLOW, TC>(a, nsm, smem, s, launched, cap);
        case 4: return launch_seg_rt<4, FLOW, TC>(a, nsm, smem, s, launched, cap);
        case 8: return launch_seg_rt<8, FLOW, TC>(a, nsm, smem, s, launched, cap);
        case 16: return launch_seg_rt<16, FLOW, TC>(a, nsm, smem, s, launched, cap);
        default: return launch_seg_rt<32, FLOW, TC>(a, nsm, smem, s, launched, cap);
    }
}

template <bool FLOW>
cudaError_t launch_seg(const KArgs& a, int rt, int nsm, size_t smem, cudaStream_t s, int* launched,
                       int cap = 0) {
    return a.tc ? launch_seg_tc<FLOW, true>(a, rt, nsm, smem, s, launched, cap)
                : launch_seg_tc<FLOW, false>(a, rt, nsm, smem, s, launched, cap);
}

template <class T>
int upload_vec(const std::vector<T>& v, T** d) {
    H2_CUDA_TRY(cudaMalloc((void**)d, sizeof(T) * std::max<size_t>(1, v.size())));
    if (!v.empty()) H2_CUDA_TRY(cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return H2_OK;
}

// Tensor-core operand buffers of an operator: the lo parts of one TF32 chunk,
// and B for the largest chunk of products of at most rt right-hand sides:
// stage_bytes / (4 * 64) K rows (a tile of at least 64 rows, 4 bytes per
// entry) x (rt rounded up to 16) columns per vector part (TF32: hi, lo; BF16:
// hi, mid, lo).
static int tc_parts_of(const h2_handle* op) { return op->params.precision == H2_BF16X3 ? 3 : 2; }
static int tc_alo_bytes(const h2_handle* op) { return op->params.precision == H2_TF32X3 ? op->stage_bytes : 0; }
static int tc_b_bytes(const h2_handle* op, int rt) {
    const int p = op->params.precision;
    if (p != H2_TF32X3 && p != H2_BF16X3) return 0;
    const int np = (std::min(rt, H2_MAX_RHS) + 15) / 16 * 16;
    return op->stage_bytes / (4 * 64) * np * (p == H2_TF32X3 ? 4 : 2) * tc_parts_of(op);
}

// Shared memory of the segment kernel with `sets` tensor-core operand sets of
// `alo` + `b` bytes.
static size_t seg_smem_raw(int rt, int stages, int stage_bytes, int alo, int b, int sets,
                           size_t xin = 0 /* 0: xin_bytes(rt) */) {
    const size_t S = (size_t)stages;
    if (xin == 0) xin = xin_bytes(rt);
    const size_t red = (size_t)kRedBuffers * sizeof(double) * kConsumers * red_rhs(rt);
    const size_t tc = (size_t)sets * ((size_t)alo + (size_t)b);
    const size_t mid = red + tc;
    return S * (size_t)stage_bytes + S * xin + mid + sizeof(uint64_t) * (2 * S + 5);
}

// Shared-memory stages of the segment kernel for r <= rt right-hand sides.
// Small r: two 32 KB stages, so that three CTAs share an SM (measured faster
// than three stages with two CTAs).  Large r (one CTA per SM): as many stages
// as fit (up to kMaxStages), so that the next chunks' copies are in flight
// while a chunk is multiplied and its predecessor's tensor-core products end.
int stages_for(int rt, int stage_bytes, int alo, int b) {
    if (rt <= 8) return 2;
    int S = 2;
    while (S < kMaxStages && seg_smem_raw(rt, S + 1, stage_bytes, alo, b, 1) <= (size_t)220 * 1024) ++S;
    return S;
}

// Two operand sets (chunk n+1 is prepared while the tensor core multiplies
// chunk n) when they fit in a CTA's shared memory, else one.
static int tc_sets_raw(int rt, int stages, int stage_bytes, int alo, int b) {
    return seg_smem_raw(rt, stages, stage_bytes, alo, b, 2) <= (size_t)220 * 1024 ? 2 : 1;
}
static size_t seg_smem_bytes(const h2_handle* op, int rt, int sets) {
    return seg_smem_raw(rt, op_stages(op, rt), op->stage_bytes, tc_alo_bytes(op), tc_b_bytes(op, rt), sets);
}
// Tensor-core tiles multiplied on the CUDA cores: at most kTcCudaMaxRT
// right-hand sides (the autotuner may turn it off).
static bool tc_cuda_for(const h2_handle* op, int rt) {
    const int p = op->params.precision;
    return (p == H2_TF32X3 || p == H2_BF16X3) && rt <= kTcCudaMaxRT && op->tc_small_r_cuda;
}
static int tc_sets_for(const h2_handle* op, int rt) {
    if (tc_cuda_for(op, rt)) return 0;   // no tensor-core operands
    return tc_sets_raw(rt, op_stages(op, rt), op->stage_bytes, tc_alo_bytes(op), tc_b_bytes(op, rt));
}

// ---- split form: shared memory of its two launches ----
// near-field launch: two stages of matrices and FP64 inputs, 2 x 2 mbarriers
static size_t near_smem_bytes(const h2_handle* op, int rt) {
    return 2 * ((size_t)op->stage_bytes + xin_bytes(rt)) + 4 * sizeof(uint64_t);
}
// far-field launch: three stages with one tensor-core operand set when both
// launches still fit one SM's shared memory (static parts and reserve aside),
// else two stages with two sets or one (measured: the third stage in flight
// is worth more than the second set).  Its chunks all have FP32 inputs (the
// near field is the other launch), so its input buffers hold FP32 rows,
// which is what lets the BF16 hi + lo far field take the third stage.
struct FarCfg {
    int stages, sets;
};
static FarCfg split_far_cfg(const h2_handle* op, int rt) {
    const size_t budget = (size_t)227 * 1024 - near_smem_bytes(op, rt) - (size_t)8 * 1024;
    const int alo = tc_alo_bytes(op), b = tc_b_bytes(op, rt);
    const size_t xin = xin_bytes_f32(rt);   // no FP64 inputs without the near field
    if (seg_smem_raw(rt, 3, op->stage_bytes, alo, b, 1, xin) <= budget) return FarCfg{3, 1};
    if (seg_smem_raw(rt, 2, op->stage_bytes, alo, b, 2, xin) <= budget) return FarCfg{2, 2};
    return FarCfg{2, 1};
}
static size_t split_far_smem(const h2_handle* op, int rt) {
    const FarCfg c = split_far_cfg(op, rt);
    return seg_smem_raw(rt, c.stages, op->stage_bytes, tc_alo_bytes(op), tc_b_bytes(op, rt), c.sets,
                        xin_bytes_f32(rt));
}

// Profiling aid (h2_profile_enable): records a CUDA event before and after
// each kernel launch of a product, on the stream the kernel is launched on,
// with what the launch computes.  A recorder without an output does nothing.
struct Prof {
    std::vector<ProfLaunch>* out = nullptr;
    std::vector<cudaEvent_t>* pool = nullptr;
    cudaError_t event(cudaEvent_t* e) {
        if (!pool->empty()) {
            *e = pool->back();
            pool->pop_back();
            return cudaSuccess;
        }
        return cudaEventCreate(e);
    }
    // Opens a launch on stream s (*idx = -1 when not recording).
    cudaError_t begin(cudaStream_t s, int* idx) {
        *idx = -1;
        if (!out) return cudaSuccess;
        ProfLaunch L;
        cudaError_t e = event(&L.e0);
        if (e == cudaSuccess) e = event(&L.e1);
        if (e != cudaSuccess) return e;
        out->push_back(L);
        *idx = (int)out->size() - 1;
        return cudaEventRecord(L.e0, s);
    }
    cudaError_t end(int idx, cudaStream_t s, int kind, int64_t bytes, int64_t macs, int grid, int r) {
        if (!out || idx < 0) return cudaSuccess;
        ProfLaunch& L = (*out)[(size_t)idx];
        L.kind = kind;
        L.bytes = bytes;
        L.macs = macs;
        L.grid = grid;
        L.r = r;
        return cudaEventRecord(L.e1, s);
    }
};

template <int RT, bool PAIR>
cudaError_t launch_near_rt(const NArgs& a, int nsm, size_t smem, cudaStream_t s) {
    cudaError_t e = set_smem(k_near_items<RT, PAIR>, smem);
    if (e != cudaSuccess) return e;
    k_near_items<RT, PAIR><<<nsm, near_cons<PAIR>() + 32, smem, s>>>(a);
    return cudaGetLastError();
}

// The split form's launches after the gather: the near field on the
// operator's second stream and the rest of the product on `s`, joined by an
// addition (u2 += u2n).
static int launch_split(h2_handle* op, double* u2, int r, int rt, cudaStream_t s, double* ws, float* ws32,
                        Prof& prof) {
    const int64_t N = op->geom->N;
    H2_CUDA_TRY(cudaMemsetAsync(u2, 0, sizeof(double) * (size_t)r * N, s));   // the expansions add into u2
    H2_CUDA_TRY(cudaMemsetAsync(op->d_u2n, 0, sizeof(double) * (size_t)r * N, s));   // the near-field units too
    H2_CUDA_TRY(cudaEventRecord(op->ev_fork, s));
    H2_CUDA_TRY(cudaStreamWaitEvent(op->near_stream, op->ev_fork, 0));
    const Pass* np = nullptr;
    for (const Pass& p : op->passes)
        if (p.kind == PASS_LEAF_NEAR) np = &p;
    if (!np) return H2_ERR_INVALID_ARG;
    NArgs na{};
    na.seg = np->d_seg;
    na.chunk = np->d_chunk;
    na.piece = np->d_piece;
    na.units = op->d_near_units;
    na.nunits = (int)op->near_units.size();
    const bool pair = op->d_near_pair != nullptr;   // paired near field (blocks and inputs)
    na.arena = pair ? reinterpret_cast<const unsigned char*>(op->d_near_pair) : op->d_arena;
    na.src_base = pair ? op->near_lo : 0;
    na.xsrc = pair ? reinterpret_cast<const unsigned char*>(op->d_wsp) : reinterpret_cast<const unsigned char*>(ws);
    na.u2n = op->d_u2n;
    na.perm = op->d_perm;
    na.N = N;
    na.r = r;
    na.stages = 2;
    na.stage_bytes = op->stage_bytes;
    na.ticket = op->d_fcnt + 3 * op->nc + 1;
    na.err = op->d_err;
    const size_t nsmem = near_smem_bytes(op, rt);
    if (rt != 16) return H2_ERR_INVALID_ARG;   // split products have 9..16 right-hand sides
    int pn = -1, pf = -1, pa = -1;
    H2_CUDA_TRY(prof.begin(op->near_stream, &pn));
    if (pair) H2_CUDA_TRY((launch_near_rt<16, true>(na, op->nsm, nsmem, op->near_stream)));
    else H2_CUDA_TRY((launch_near_rt<16, false>(na, op->nsm, nsmem, op->near_stream)));
    H2_CUDA_TRY(prof.end(pn, op->near_stream, PASS_SPLIT_NEAR, np->bytes, np->macs, op->nsm, r));
    KArgs a{};
    a.nops = 1;
    a.ctx[0] = OpCtx{op->d_arena, ws, ws32, u2, op->d_perm, N, r, op->kp, op->d_nodes, op->row_yhat};
    a.err = op->d_err;
    a.r = r;
    const FarCfg fc = split_far_cfg(op, rt);
    a.stages = fc.stages;
    a.stage_bytes = op->stage_bytes;
    a.xin_bytes = (int)xin_bytes_f32(rt);
    a.tc = op->params.precision == H2_TF32X3 || op->params.precision == H2_BF16X3;
    a.tc_alo_bytes = tc_alo_bytes(op);
    a.tc_b_bytes = tc_b_bytes(op, rt);
    a.tc_parts = tc_parts_of(op);
    a.tc_sets = fc.sets;
    a.seg = op->d_sseg;
    a.chunk = op->d_schunk;
    a.piece = op->d_spiece;
    a.deps = op->d_sdeps;
    a.expect = op->d_sexpect;
    a.cnt = op->d_fcnt;
    a.nseg = (int)op->split.seg.size();
    a.nreg = 3 * op->nc;
    // one CTA per SM, so that a near-field CTA fits beside it
    H2_CUDA_TRY(prof.begin(s, &pf));
    H2_CUDA_TRY(launch_seg<true>(a, rt, op->nsm, split_far_smem(op, rt), s, &op->flow_grid, 1));
    H2_CUDA_TRY(prof.end(pf, s, PASS_SPLIT_FAR, op->bytes_streamed - np->bytes, op->macs - np->macs, op->flow_grid, r));
    H2_CUDA_TRY(cudaEventRecord(op->ev_join, op->near_stream));
    H2_CUDA_TRY(cudaStreamWaitEvent(s, op->ev_join, 0));
    const int64_t n = (int64_t)r * N;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * (int64_t)op->nsm));
    H2_CUDA_TRY(prof.begin(s, &pa));
    k_add<<<grid, 256, 0, s>>>(u2, op->d_u2n, n);
    H2_CUDA_TRY(cudaGetLastError());
    H2_CUDA_TRY(prof.end(pa, s, PASS_SPLIT_ADD, 0, 0, grid, r));
    return H2_OK;
}

static bool split_active(const h2_handle* op, bool flow, int rt) {
    return flow && op->has_split && op->use_split && rt > 8;
}

// Kernel launches of one product with max_rhs right-hand sides.
static int launches_per_matvec(const h2_handle* op) {
    if (!op->use_flow) return 1 + (int)op->passes.size();
    const int r = op->params.max_rhs;
    if (!split_active(op, true, rt_for(r))) return 2;
    // products of at most 16 right-hand sides: 4 launches each (a rest of at
    // most 8 is one single-launch product: 2)
    const int rest = r % 16;
    return 4 * (r / 16) + (rest == 0 ? 0 : rest > 8 ? 4 : 2);
}

// Launches the gather kernel and every pass (level-wise) or the flow kernel
// on workspaces `ws` (FP64) and `ws32` (FP32 operators only).
int launch_matvec(h2_handle* op, const double* u1, double* u2, int r, cudaStream_t s, double* ws,
                  float* ws32, bool flow, std::vector<ProfLaunch>* prof_out,
                  std::vector<cudaEvent_t>* pool) {
    if (r > 16 && split_active(op, flow, rt_for(r))) {
        // the split form in products of at most 16 right-hand sides: at 32 a
        // far-field CTA (168 registers per thread) leaves no SM sub-partition
        // room for a near-field warp, at 16 both fit
        for (int c0 = 0; c0 < r; c0 += 16) {
            const int rc = launch_matvec(op, u1 + (int64_t)c0 * op->geom->N, u2 + (int64_t)c0 * op->geom->N,
                                         std::min(16, r - c0), s, ws, ws32, flow, prof_out, pool);
            if (rc != H2_OK) return rc;
        }
        return H2_OK;
    }
    const int rt = rt_for(r);
    if ((int64_t)op->chunk_cols * r > (int64_t)xin_cols(rt) * rt) return H2_ERR_INVALID_ARG;   // stage inputs
    const size_t smem = pass_smem_bytes(op, rt);
    const int64_t N = op->geom->N;
    Prof prof{prof_out, pool};
    int pi = -1;
    H2_CUDA_TRY(prof.begin(s, &pi));
    const bool split = split_active(op, flow, rt);
    int gather_grid = 0;
    {
        const std::vector<int32_t>& zr = split ? op->split.zero_rows[0] : flow ? op->fzero_rows : op->zero_rows;
        const int32_t* d_zr = split ? op->d_szero_rows : flow ? op->d_fzero_rows : op->d_zero_rows;
        const int nclear = flow ? 3 * op->nc + 2 : 0;
        const int64_t work = std::max<int64_t>({op->row_xhat * r, (int64_t)zr.size() * op->kp * r, (int64_t)nclear});
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096));
        float2* wsp = split && op->d_near_pair ? op->d_wsp : nullptr;
        k_prologue<<<grid, 256, 0, s>>>(u1, ws, ws32, wsp, op->d_gather_src, op->row_xhat, N, r, d_zr, (int)zr.size(),
                                        op->kp, op->d_fcnt, nclear);
        H2_CUDA_TRY(cudaGetLastError());
        gather_grid = grid;
    }
    H2_CUDA_TRY(prof.end(pi, s, PASS_PROLOGUE, 0, 0, gather_grid, r));
    if (split) return launch_split(op, u2, r, rt, s, ws, ws32, prof);
    KArgs a{};
    a.nops = 1;
    a.ctx[0] = OpCtx{op->d_arena, ws, ws32, u2, op->d_perm, N, r, op->kp, op->d_nodes, op->row_yhat};
    a.err = op->d_err;
    a.r = r;
    a.stages = op_stages(op, rt);
    a.stage_bytes = op->stage_bytes;
    a.xin_bytes = (int)xin_bytes(rt);
    a.tc = (op->params.precision == H2_TF32X3 || op->params.precision == H2_BF16X3) && !tc_cuda_for(op, rt);
    a.tc_alo_bytes = tc_alo_bytes(op);
    a.tc_b_bytes = tc_b_bytes(op, rt);
    a.tc_parts = tc_parts_of(op);
    a.tc_sets = tc_sets_for(op, rt);
    a.tc_cuda = tc_cuda_for(op, rt) ? 1 : 0;
    if (flow) {
        a.seg = op->d_fseg;
        a.chunk = op->d_fchunk;
        a.piece = op->d_fpiece;
        a.deps = op->d_fdeps;
        a.expect = op->d_fexpect;
        a.cnt = op->d_fcnt;
        a.nseg = (int)op->fseg.size();
        a.nreg = 3 * op->nc;
        H2_CUDA_TRY(prof.begin(s, &pi));
        H2_CUDA_TRY(launch_seg<true>(a, rt, op->nsm, smem, s, &op->flow_grid, op->tune_ctas));
        H2_CUDA_TRY(prof.end(pi, s, PASS_FLOW, op->bytes_streamed, op->macs, op->flow_grid, r));
        return H2_OK;
    }
    for (Pass& p : op->passes) {
        a.seg = p.d_seg;
        a.chunk = p.d_chunk;
        a.piece = p.d_piece;
        a.nseg = (int)p.seg.size();
        H2_CUDA_TRY(prof.begin(s, &pi));
        H2_CUDA_TRY(launch_seg<false>(a, rt, op->nsm, smem, s, &p.grid, op->tune_ctas));
        H2_CUDA_TRY(prof.end(pi, s, p.kind, p.bytes, p.macs, p.grid, r));
    }
    return H2_OK;
}

}  // namespace

size_t pass_smem_bytes(const h2_handle* op, int rt) { return seg_smem_bytes(op, rt, tc_sets_for(op, rt)); }

// Resident CTAs and per-CTA rates of the dataflow kernel on the current
// device for the operator's largest r (input of the ticket-order simulation).
static int flow_model_raw(int rt, bool tc, size_t smem, int r, FlowModel& fm, int cap = 0) {
    int dev = 0, nsm = 0, khz = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    H2_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    H2_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    int occ = 1;
    switch (rt) {
        case 1: occ = tc ? seg_occupancy<1, true>(smem) : seg_occupancy<1, false>(smem); break;
        case 2: occ = tc ? seg_occupancy<2, true>(smem) : seg_occupancy<2, false>(smem); break;
        case 4: occ = tc ? seg_occupancy<4, true>(smem) : seg_occupancy<4, false>(smem); break;
        case 8: occ = tc ? seg_occupancy<8, true>(smem) : seg_occupancy<8, false>(smem); break;
        case 16: occ = tc ? seg_occupancy<16, true>(smem) : seg_occupancy<16, false>(smem); break;
        default: occ = tc ? seg_occupancy<32, true>(smem) : seg_occupancy<32, false>(smem); break;
    }
    const double ghz = khz > 0 ? khz * 1e-6 : 2.07;
    if (cap > 0 && cap < occ) occ = cap;
    fm.workers = nsm * occ;
    fm.r = r;
    fm.f64_per_ns = 2.0 * ghz / occ;
    fm.f32_per_ns = 128.0 * ghz / occ;
    fm.bytes_per_ns = 6800.0 / fm.workers;
    return H2_OK;
}

int flow_model(h2_handle* op, FlowModel& fm) {
    const int rt = rt_for(op->params.max_rhs);
    const bool tc = (op->params.precision == H2_TF32X3 || op->params.precision == H2_BF16X3) && !tc_cuda_for(op, rt);
    return flow_model_raw(rt, tc, pass_smem_bytes(op, rt), op->params.max_rhs, fm, op->tune_ctas);
}

// The split form applies to FP32 and BF16 hi+lo operators built for more than
// 8 right-hand sides whose leaves have at most 64 rows (the near-field
// kernel's work items: 64 rows x r over 128 threads, r / 2 per thread).
bool split_possible(const h2_handle* op) {
    const int p = op->params.precision;
    if ((p != H2_FP32 && p != H2_BF16X3) || op->params.max_rhs <= 8) return false;
    bool near = false;
    for (const Pass& q : op->passes)
        if (q.kind == PASS_LEAF_NEAR) {
            near = true;
            for (const Segment& sg : q.seg)
                if (sg.nrows > 64) return false;
        }
    return near;
}

int build_split(h2_handle* op) {
    op->has_split = 0;
    if (!split_possible(op)) return H2_OK;
    const int rt = rt_for(op->params.max_rhs);
    const bool tc = op->params.precision == H2_BF16X3;
    FlowModel fm;
    const int rc = flow_model_raw(rt, tc, split_far_smem(op, rt), op->params.max_rhs, fm, 1);
    if (rc != H2_OK) return rc;
    if (build_flow_multi({op}, fm, op->split, true) < 0.0) return H2_OK;   // single launch only
    // near-field work units: runs of at most `maxc` chunks of a segment, so
    // that there are about 8 units per SM; longest first
    const Pass* np = nullptr;
    for (const Pass& p : op->passes)
        if (p.kind == PASS_LEAF_NEAR) np = &p;
    int64_t total = 0;
    for (const Segment& sg : np->seg) total += sg.nchunks;
    const int maxc = (int)std::max<int64_t>(2, (total + 8LL * fm.workers - 1) / (8LL * fm.workers));
    op->near_units.clear();
    for (size_t i = 0; i < np->seg.size(); ++i) {
        const int nch = np->seg[i].nchunks;
        const int parts = (nch + maxc - 1) / maxc;
        for (int q = 0; q < parts; ++q) {
            const int c0 = (int)((int64_t)nch * q / parts), c1 = (int)((int64_t)nch * (q + 1) / parts);
            op->near_units.push_back({(int32_t)i, c0, c1 - c0, 0});
        }
    }
    std::stable_sort(op->near_units.begin(), op->near_units.end(),
                     [](const std::array<int32_t, 4>& x, const std::array<int32_t, 4>& y) { return x[2] > y[2]; });
    op->has_split = 1;
    return H2_OK;
}

// Checks, on the host, the invariants the bulk copies rely on (16-byte aligned
// sources, destinations and sizes; chunks within one stage; input rows on
// 4-row boundaries), so that a plan that violates them is rejected before any
// kernel sees it.
static int validate_chunks(const h2_handle* op, const std::vector<Segment>* segs, const std::vector<Chunk>& chunks,
                           const std::vector<Piece>& pieces) {
    for (const Chunk& c : chunks) {
        if (c.src % 16 || c.bytes % 16 || c.bytes <= 0 || c.bytes > op->stage_bytes || c.npieces < 1 ||
            c.npieces > H2_MAX_CHUNK_PIECES || c.ncols < 1 || c.ncols > op->chunk_cols ||
            c.src + c.bytes > op->arena_bytes || (size_t)c.piece0 + c.npieces > pieces.size())
            return H2_ERR_INVALID_ARG;
        int cols = 0;
        for (int q = 0; q < c.npieces; ++q) {
            const Piece& p = pieces[(size_t)c.piece0 + q];
            if (p.in_row % 4 || p.in_row < 0 || p.smem_off % 16 || p.smem_off >= c.bytes ||
                (int64_t)p.in_row + p.ncols > op->ws_rows - 4)
                return H2_ERR_INVALID_ARG;
            cols += p.ncols;
        }
        if (cols != c.ncols || pieces[c.piece0].in_row != c.in_row0 || pieces[c.piece0].type != c.type0)
            return H2_ERR_INVALID_ARG;
        for (int q = 1; q < c.npieces; ++q)   // one piece type per chunk
            if (pieces[(size_t)c.piece0 + q].type != c.type0) return H2_ERR_INVALID_ARG;
    }
    if (segs)
        for (const Segment& sg : *segs) {
            if (sg.nchunks < 1 || sg.nrows < 1 || sg.nrows > H2_MAX_LEAF || (size_t)sg.chunk0 + sg.nchunks > chunks.size())
                return H2_ERR_INVALID_ARG;
            // the consumers keep one kind of accumulator per segment: tensor
            // memory or registers, and packed FP32 sums when the output is FP32
            const bool tc0 = piece_tc(chunks[sg.chunk0].type0);
            for (int q = 0; q < sg.nchunks; ++q) {
                const int t = chunks[(size_t)sg.chunk0 + q].type0;
                if (piece_tc(t) != tc0 || (sg.out_f32 && t == PIECE_F64)) return H2_ERR_INVALID_ARG;
            }
        }
    return H2_OK;
}

// (Re)uploads the dataflow arrays of an operator (its ticket order may have
// been rebuilt by the autotuner).
static int upload_flow(h2_handle* op) {
    for (void** p : {(void**)&op->d_fseg, (void**)&op->d_fchunk, (void**)&op->d_fpiece, (void**)&op->d_fdeps,
                     (void**)&op->d_fexpect, (void**)&op->d_fzero_rows})
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    int rc;
    if ((rc = upload_vec(op->fseg, &op->d_fseg)) || (rc = upload_vec(op->fchunk, &op->d_fchunk)) ||
        (rc = upload_vec(op->fpiece, &op->d_fpiece)) || (rc = upload_vec(op->fdeps, &op->d_fdeps)) ||
        (rc = upload_vec(op->fexpect, &op->d_fexpect)) || (rc = upload_vec(op->fzero_rows, &op->d_fzero_rows)))
        return rc;
    if (!op->d_fcnt) H2_CUDA_TRY(cudaMalloc((void**)&op->d_fcnt, sizeof(int32_t) * (3 * (size_t)op->nc + 2)));
    return H2_OK;
}

int upload_plan(h2_handle* op) {
    for (const Pass& p : op->passes) {
        if (validate_chunks(op, &p.seg, p.chunk, p.piece) != H2_OK) {
            set_last_error("h2_assemble: internal plan check failed (bulk-copy alignment or chunk limits)");
            return H2_ERR_INVALID_ARG;
        }
    }
    if (op->use_flow && validate_chunks(op, nullptr, op->fchunk, op->fpiece) != H2_OK) {
        set_last_error("h2_assemble: internal plan check failed (dataflow chunks)");
        return H2_ERR_INVALID_ARG;
    }
    int dev = 0, nsm = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    H2_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int rc;
    for (Pass& p : op->passes) {
        std::vector<FlowSeg> fs(p.seg.size());
        for (size_t i = 0; i < p.seg.size(); ++i) fs[i] = FlowSeg{p.seg[i], -1, 0, 0, p.kind, 0, 0};
        if ((rc = upload_vec(fs, &p.d_seg)) || (rc = upload_vec(p.chunk, &p.d_chunk)) ||
            (rc = upload_vec(p.piece, &p.d_piece)))
            return rc;
        p.grid = 0;
    }
    op->nsm = nsm;
    if ((rc = upload_vec(op->zero_rows, &op->d_zero_rows))) return rc;
    if (op->use_flow && (rc = upload_flow(op))) return rc;
    if (op->has_split) {
        if (validate_chunks(op, nullptr, op->split.chunk, op->split.piece) != H2_OK) {
            set_last_error("h2_assemble: internal plan check failed (split dataflow chunks)");
            return H2_ERR_INVALID_ARG;
        }
        if ((rc = upload_vec(op->split.seg, &op->d_sseg)) || (rc = upload_vec(op->split.chunk, &op->d_schunk)) ||
            (rc = upload_vec(op->split.piece, &op->d_spiece)) || (rc = upload_vec(op->split.deps, &op->d_sdeps)) ||
            (rc = upload_vec(op->split.expect, &op->d_sexpect)) ||
            (rc = upload_vec(op->split.zero_rows[0], &op->d_szero_rows)))
            return rc;
        if (!op->d_fcnt) H2_CUDA_TRY(cudaMalloc((void**)&op->d_fcnt, sizeof(int32_t) * (3 * (size_t)op->nc + 2)));
        H2_CUDA_TRY(cudaMalloc((void**)&op->d_u2n, sizeof(double) * (size_t)op->params.max_rhs * op->geom->N));
        H2_CUDA_TRY(cudaMalloc((void**)&op->d_near_units, sizeof(int4) * std::max<size_t>(1, op->near_units.size())));
        H2_CUDA_TRY(cudaMemcpy(op->d_near_units, op->near_units.data(), sizeof(int4) * op->near_units.size(),
                               cudaMemcpyHostToDevice));
        H2_CUDA_TRY(cudaStreamCreateWithFlags(&op->near_stream, cudaStreamNonBlocking));
        H2_CUDA_TRY(cudaEventCreateWithFlags(&op->ev_fork, cudaEventDisableTiming));
        H2_CUDA_TRY(cudaEventCreateWithFlags(&op->ev_join, cudaEventDisableTiming));
        if (op->params.near_field == H2_NEAR_F32PAIR) {
            // the near pass's contiguous arena range, paired by the assembly
            const Pass* np = nullptr;
            for (const Pass& q : op->passes)
                if (q.kind == PASS_LEAF_NEAR) np = &q;
            op->near_lo = INT64_MAX;
            op->near_hi = 0;
            for (const Chunk& c : np->chunk) {
                op->near_lo = std::min<int64_t>(op->near_lo, c.src);
                op->near_hi = std::max<int64_t>(op->near_hi, c.src + c.bytes);
            }
            if (op->near_hi <= op->near_lo) op->near_lo = op->near_hi = 0;
            H2_CUDA_TRY(cudaMalloc((void**)&op->d_near_pair, (size_t)std::max<int64_t>(16, op->near_hi - op->near_lo)));
            H2_CUDA_TRY(cudaMalloc((void**)&op->d_wsp, sizeof(float2) * (size_t)op->ws_rows * op->params.max_rhs));
        }
    }
    if ((rc = upload_vec(op->gather_src, &op->d_gather_src))) return rc;
    H2_CUDA_TRY(cudaMalloc((void**)&op->d_ws, sizeof(double) * (size_t)op->ws_rows * op->params.max_rhs));
    if (op->params.precision != H2_FP64)
        H2_CUDA_TRY(cudaMalloc((void**)&op->d_ws32, sizeof(float) * (size_t)op->ws_rows * op->params.max_rhs));
    H2_CUDA_TRY(cudaMalloc((void**)&op->d_err, sizeof(int)));
    H2_CUDA_TRY(cudaMemset(op->d_err, 0, sizeof(int)));
    op->n_launches = launches_per_matvec(op);
    return H2_OK;
}

void release_graph(h2_handle* op) {
    if (op->graph_exec) cudaGraphExecDestroy(op->graph_exec);
    if (op->graph) cudaGraphDestroy(op->graph);
    op->graph_exec = nullptr;
    op->graph = nullptr;
    op->graph_r = 0;
    op->graph_u1 = nullptr;
    op->graph_u2 = nullptr;
    op->graph_seen = 0;
}

void release_profile(h2_handle* op) {
    for (auto& call : op->prof_calls)
        for (const ProfLaunch& L : call) {
            cudaEventDestroy(L.e0);
            cudaEventDestroy(L.e1);
        }
    for (cudaEvent_t e : op->prof_pool) cudaEventDestroy(e);
    op->prof_calls.clear();
    op->prof_pool.clear();
}

// Per launch of the recorded calls (launch i of every call: calls with the
// same r launch the same kernels), its description (from the first call) and
// its total time over the calls.
int read_profile(h2_handle* op, std::vector<ProfLaunch>& launches, std::vector<double>& ms, int& ncalls) {
    launches.clear();
    ms.clear();
    ncalls = (int)op->prof_calls.size();
    int rc = H2_OK;
    for (auto& call : op->prof_calls) {
        if (launches.empty()) launches = call;
        if (ms.size() < call.size()) ms.resize(call.size(), 0.0);
        for (size_t i = 0; i < call.size(); ++i) {
            float t = 0.0f;
            cudaError_t e = cudaEventSynchronize(call[i].e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, call[i].e0, call[i].e1);
            if (e != cudaSuccess && rc == H2_OK) {
                set_cuda_error(e, "cudaEventElapsedTime", __FILE__, __LINE__);
                rc = H2_ERR_CUDA;
            }
            ms[i] += t;
        }
    }
    for (auto& call : op->prof_calls)
        for (const ProfLaunch& L : call) {
            op->prof_pool.push_back(L.e0);
            op->prof_pool.push_back(L.e1);
        }
    op->prof_calls.clear();
    return rc;
}

// One product on device buffers.  A product with the same (u1, u2, r) as the
// previous call is captured into a CUDA graph (on the operator's own capture
// stream) and replayed from then on; products while the caller's stream is
// itself being captured, while profiling, or after a failed capture are
// launched directly.
int matvec_device(h2_handle* op, const double* u1, double* u2, int r, cudaStream_t s) {
    if (op->prof_enabled) {
        std::vector<ProfLaunch> ev;
        int rc = launch_matvec(op, u1, u2, r, s, op->d_ws, op->d_ws32, op->use_flow != 0, &ev, &op->prof_pool);
        op->prof_calls.push_back(std::move(ev));
        return rc;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    if (cs == cudaStreamCaptureStatusNone && !op->graph_fail) {
        const bool same = op->graph_u1 == u1 && op->graph_u2 == u2 && op->graph_r == r;
        if (same && op->graph_exec) {
            H2_CUDA_TRY(cudaGraphLaunch(op->graph_exec, s));
            return H2_OK;
        }
        if (same && op->graph_seen > 0) {
            bool ok = true;
            if (!op->capture_stream)
                ok = cudaStreamCreateWithFlags(&op->capture_stream, cudaStreamNonBlocking) == cudaSuccess;
            ok = ok && cudaStreamBeginCapture(op->capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            int rc = H2_ERR_CUDA;
            if (ok) {
                rc = launch_matvec(op, u1, u2, r, op->capture_stream, op->d_ws, op->d_ws32, op->use_flow != 0,
                                   nullptr, nullptr);
                cudaGraph_t g = nullptr;
                ok = cudaStreamEndCapture(op->capture_stream, &g) == cudaSuccess && rc == H2_OK && g;
                if (ok) ok = cudaGraphInstantiate(&op->graph_exec, g, 0) == cudaSuccess;
                if (ok) op->graph = g;
                else if (g) cudaGraphDestroy(g);
            }
            if (ok) {
                H2_CUDA_TRY(cudaGraphLaunch(op->graph_exec, s));
                return H2_OK;
            }
            cudaGetLastError();   // capture did not work here: direct launches from now on
            op->graph_exec = nullptr;
            op->graph_fail = 1;
        } else if (!same) {
            release_graph(op);
            op->graph_u1 = u1;
            op->graph_u2 = u2;
            op->graph_r = r;
            op->graph_seen = 1;
        }
    }
    return launch_matvec(op, u1, u2, r, s, op->d_ws, op->d_ws32, op->use_flow != 0, nullptr, nullptr);
}

// The largest dynamic shared memory one segment-kernel CTA can be given: the
// device's per-block opt-in limit less the kernel's static shared memory (the
// same for every instantiation).
static size_t seg_smem_max() {
    static size_t v = 0;
    if (v == 0) {
        int dev = 0, optin = 0;
        cudaFuncAttributes fa{};
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, k_seg<32, true, true>) == cudaSuccess && optin > (int)fa.sharedSizeBytes) {
            v = (size_t)optin - fa.sharedSizeBytes;
        } else {
            cudaGetLastError();
            v = (size_t)220 * 1024;
        }
    }
    return v;
}

// Times one configuration: `iters` products after two unmeasured ones.
static int time_products(h2_handle* op, const double* x, double* y, int r, cudaStream_t s, int iters,
                         double* ms) {
    for (int i = 0; i < 2; ++i) {
        int rc = launch_matvec(op, x, y, r, s, op->d_ws, op->d_ws32, op->use_flow != 0, nullptr, nullptr);
        if (rc != H2_OK) return rc;
    }
    cudaEvent_t e0, e1;
    H2_CUDA_TRY(cudaEventCreate(&e0));
    H2_CUDA_TRY(cudaEventCreate(&e1));
    H2_CUDA_TRY(cudaEventRecord(e0, s));
    int rc = H2_OK;
    for (int i = 0; i < iters && rc == H2_OK; ++i)
        rc = launch_matvec(op, x, y, r, s, op->d_ws, op->d_ws32, op->use_flow != 0, nullptr, nullptr);
    H2_CUDA_TRY(cudaEventRecord(e1, s));
    H2_CUDA_TRY(cudaEventSynchronize(e1));
    float t = 0.0f;
    H2_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = (double)t / iters;
    return rc;
}

// Ticket order of the dataflow form for the operator's current launch
// configuration, uploaded.
static int rebuild_flow(h2_handle* op) {
    FlowModel fm;
    int rc = flow_model(op, fm);
    if (rc != H2_OK) return rc;
    if (build_flow(op, fm) < 0.0) return H2_ERR_INVALID_ARG;
    return upload_flow(op);
}

int autotune(h2_handle* op, int r, cudaStream_t s, h2_tuning_t* out) {
    const int64_t N = op->geom->N;
    double *x = nullptr, *y = nullptr;
    H2_CUDA_TRY(cudaMalloc((void**)&x, sizeof(double) * (size_t)N * r));
    H2_CUDA_TRY(cudaMalloc((void**)&y, sizeof(double) * (size_t)N * r));
    H2_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * (size_t)N * r, s));
    release_graph(op);
    const bool have_flow = !op->fseg.empty();
    const int use_flow0 = op->use_flow, st0 = op->tune_stages, ct0 = op->tune_ctas;
    double ms0 = 0.0;
    int rc = time_products(op, x, y, r, s, 1, &ms0);
    const int iters = std::max(1, std::min(10, (int)(20.0 / std::max(ms0, 1e-3))));
    if (rc == H2_OK) rc = time_products(op, x, y, r, s, iters, &ms0);
    int best_flow = use_flow0, best_st = st0, best_ct = ct0, ncand = 0;
    const int rt = rt_for(r);
    const bool can_split = op->has_split && rt > 8;
    int best_split = op->use_split;
    double best = ms0;
    const bool tc = (op->params.precision == H2_TF32X3 || op->params.precision == H2_BF16X3) && !tc_cuda_for(op, rt);
    for (int flow = have_flow ? 1 : 0; flow >= 0 && rc == H2_OK; --flow) {
        for (int stages = 2; stages <= 4 && rc == H2_OK; ++stages) {
            op->tune_stages = stages;
            const size_t smem = pass_smem_bytes(op, rt);
            if (smem > seg_smem_max()) continue;
            int occ = 1;
            switch (rt) {
                case 1: occ = tc ? seg_occupancy<1, true>(smem) : seg_occupancy<1, false>(smem); break;
                case 2: occ = tc ? seg_occupancy<2, true>(smem) : seg_occupancy<2, false>(smem); break;
                case 4: occ = tc ? seg_occupancy<4, true>(smem) : seg_occupancy<4, false>(smem); break;
                case 8: occ = tc ? seg_occupancy<8, true>(smem) : seg_occupancy<8, false>(smem); break;
                case 16: occ = tc ? seg_occupancy<16, true>(smem) : seg_occupancy<16, false>(smem); break;
                default: occ = tc ? seg_occupancy<32, true>(smem) : seg_occupancy<32, false>(smem); break;
            }
            for (int cap = 1; cap <= std::min(occ, 4) && rc == H2_OK; ++cap) {
                op->tune_ctas = cap;
                op->use_flow = flow;
                op->use_split = 0;
                if (flow && (rc = rebuild_flow(op)) != H2_OK) break;
                double ms = 0.0;
                rc = time_products(op, x, y, r, s, iters, &ms);
                ++ncand;
                if (rc == H2_OK && ms < best) {
                    best = ms;
                    best_flow = flow;
                    best_st = stages;
                    best_ct = cap;
                    best_split = 0;
                }
            }
        }
    }
    if (can_split && rc == H2_OK) {   // the split form (its own stage and CTA counts)
        op->use_flow = 1;
        op->use_split = 1;
        double ms = 0.0;
        rc = time_products(op, x, y, r, s, iters, &ms);
        ++ncand;
        if (rc == H2_OK && ms < best) {
            best = ms;
            best_flow = 1;
            best_split = 1;
        }
    }
    op->use_split = best_split;
    // tensor-core tiles on the CUDA cores or on the tensor cores (small r)
    const int prec = op->params.precision;
    if (rc == H2_OK && (prec == H2_TF32X3 || prec == H2_BF16X3) && rt <= kTcCudaMaxRT) {
        const int cur = op->tc_small_r_cuda;
        op->use_flow = best_flow;
        op->tune_ctas = best_ct;
        op->tc_small_r_cuda = !cur;
        // the other pipe with the best stage count, or fewer stages where its
        // operand buffers (tensor-core tiles) no longer fit beside that many
        int st = best_st;
        op->tune_stages = st;
        while (st > 2 && pass_smem_bytes(op, rt) > seg_smem_max()) op->tune_stages = --st;
        double ms = 0.0;
        const bool fits = pass_smem_bytes(op, rt) <= seg_smem_max();
        if (fits) {
            rc = time_products(op, x, y, r, s, iters, &ms);
            ++ncand;
        }
        if (fits && rc == H2_OK && ms < best) {
            best = ms;
            best_st = st;
        } else {
            op->tc_small_r_cuda = cur;
        }
    }
    op->use_flow = best_flow;
    op->tune_stages = best_st;
    op->tune_ctas = best_ct;
    op->tune_ms = best;
    if (rc == H2_OK && have_flow) rc = rebuild_flow(op);   // the order for the chosen CTA count
    op->use_flow = best_flow;
    op->n_launches = launches_per_matvec(op);
    cudaFree(x);
    cudaFree(y);
    if (out) {
        out->schedule = op->use_flow ? H2_SCHEDULE_FLOW : H2_SCHEDULE_LEVELS;
        out->stages = op_stages(op, rt);
        out->ctas_per_sm = op->tune_ctas;
        out->n_candidates = ncand;
        out->ms_best = best;
        out->ms_default = ms0;
    }
    return rc;
}

// ---------------------------------------------------------------------------
// Batched product over several operators: their dataflow segments merged into
// one ticket order (list-scheduled together), one input gather per operator,
// then ONE persistent launch; every segment finds its operator's arena,
// workspaces, u2, permutation, N and r in a context table passed with the
// launch.  Merged schedules are cached per set of operators.
// ---------------------------------------------------------------------------
namespace {
struct BatchPlan {
    std::vector<uint64_t> serials;
    FlowOut fo;
    FlowSeg* d_seg = nullptr;
    Chunk* d_chunk = nullptr;
    Piece* d_piece = nullptr;
    int32_t* d_deps = nullptr;
    int32_t* d_expect = nullptr;
    int32_t* d_cnt = nullptr;
    std::vector<int32_t*> d_zero;
    int grid = 0;
    ~BatchPlan() {
        for (void* p : {(void*)d_seg, (void*)d_chunk, (void*)d_piece, (void*)d_deps, (void*)d_expect, (void*)d_cnt})
            if (p) cudaFree(p);
        for (int32_t* p : d_zero)
            if (p) cudaFree(p);
    }
};
std::mutex g_batch_mu;
std::vector<std::unique_ptr<BatchPlan>> g_batches;
}  // namespace

void drop_batch_plans(uint64_t serial) {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batches.erase(std::remove_if(g_batches.begin(), g_batches.end(),
                                   [&](const std::unique_ptr<BatchPlan>& b) {
                                       return std::find(b->serials.begin(), b->serials.end(), serial) !=
                                              b->serials.end();
                                   }),
                    g_batches.end());
}

int matvec_batched(h2_handle* const* ops, int n, const double* const* u1, double* const* u2, const int32_t* r,
                   cudaStream_t s) {
    int rmax = 1, alo = 0, b = 0, parts = 2;
    bool tc = false;
    for (int i = 0; i < n; ++i) rmax = std::max(rmax, (int)r[i]);
    for (int i = 0; i < n; ++i) {
        alo = std::max(alo, tc_alo_bytes(ops[i]));
        b = std::max(b, tc_b_bytes(ops[i], rt_for(rmax)));
        if (tc_b_bytes(ops[i], rt_for(rmax)) > 0) parts = std::max(parts, tc_parts_of(ops[i]));
        tc = tc || ops[i]->params.precision == H2_TF32X3 || ops[i]->params.precision == H2_BF16X3;
        if (ops[i]->stage_bytes != ops[0]->stage_bytes || ops[i]->device != ops[0]->device) return H2_ERR_INVALID_ARG;
    }
    const int rt = rt_for(rmax);
    const int stage_bytes = ops[0]->stage_bytes;
    const int nst = stages_for(rt, stage_bytes, alo, b);
    const bool tcc = tc && rt <= kTcCudaMaxRT;   // tensor tiles on the CUDA cores
    const int sets = tcc ? 0 : tc ? tc_sets_raw(rt, nst, stage_bytes, alo, b) : 1;
    const size_t smem = seg_smem_raw(rt, nst, stage_bytes, alo, b, sets);
    for (int i = 0; i < n; ++i)   // a stage holds every chunk's inputs
        if ((int64_t)ops[i]->chunk_cols * r[i] > (int64_t)xin_cols(rt) * rt) return H2_ERR_INVALID_ARG;
    std::vector<uint64_t> key(n);
    for (int i = 0; i < n; ++i) key[i] = ops[i]->serial;
    BatchPlan* bp = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_batch_mu);
        for (auto& p : g_batches)
            if (p->serials == key) bp = p.get();
    }
    if (!bp) {
        auto nb = std::make_unique<BatchPlan>();
        nb->serials = key;
        FlowModel fm;
        int rc = flow_model_raw(rt, tc, smem, rmax, fm);
        if (rc != H2_OK) return rc;
        if (build_flow_multi(std::vector<h2_handle*>(ops, ops + n), fm, nb->fo) < 0.0) {
            set_last_error("h2_matvec_batched: no dataflow order exists for these operators");
            return H2_ERR_INVALID_ARG;
        }
        // (the chunks are copies of the operators' own chunks, checked when each
        // operator was assembled)
        if ((rc = upload_vec(nb->fo.seg, &nb->d_seg)) || (rc = upload_vec(nb->fo.chunk, &nb->d_chunk)) ||
            (rc = upload_vec(nb->fo.piece, &nb->d_piece)) || (rc = upload_vec(nb->fo.deps, &nb->d_deps)) ||
            (rc = upload_vec(nb->fo.expect, &nb->d_expect)))
            return rc;
        H2_CUDA_TRY(cudaMalloc((void**)&nb->d_cnt, sizeof(int32_t) * ((size_t)nb->fo.nreg + 1)));
        nb->d_zero.assign(n, nullptr);
        for (int i = 0; i < n; ++i)
            if ((rc = upload_vec(nb->fo.zero_rows[i], &nb->d_zero[i]))) return rc;
        bp = nb.get();
        std::lock_guard<std::mutex> lock(g_batch_mu);
        g_batches.push_back(std::move(nb));
    }
    // gather every operator's input; the first gather also clears the counters
    for (int i = 0; i < n; ++i) {
        h2_handle* op = ops[i];
        const std::vector<int32_t>& zr = bp->fo.zero_rows[i];
        const int nclear = i == 0 ? bp->fo.nreg + 1 : 0;
        const int64_t work =
            std::max<int64_t>({op->row_xhat * r[i], (int64_t)zr.size() * op->kp * r[i], (int64_t)nclear});
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096));
        k_prologue<<<grid, 256, 0, s>>>(u1[i], op->d_ws, op->d_ws32, nullptr, op->d_gather_src, op->row_xhat, op->geom->N,
                                        r[i], bp->d_zero[i], (int)zr.size(), op->kp, bp->d_cnt, nclear);
        H2_CUDA_TRY(cudaGetLastError());
    }
    KArgs a{};
    a.nops = n;
    for (int i = 0; i < n; ++i)
        a.ctx[i] = OpCtx{ops[i]->d_arena, ops[i]->d_ws, ops[i]->d_ws32, u2[i], ops[i]->d_perm, ops[i]->geom->N,
                         (int)r[i], ops[i]->kp, ops[i]->d_nodes, ops[i]->row_yhat};
    a.err = ops[0]->d_err;
    a.r = rmax;
    a.stages = nst;
    a.stage_bytes = stage_bytes;
    a.xin_bytes = (int)xin_bytes(rt);
    a.tc = tc && !tcc;
    a.tc_alo_bytes = alo;
    a.tc_b_bytes = b;
    a.tc_parts = parts;
    a.tc_sets = sets;
    a.tc_cuda = tcc ? 1 : 0;
    a.seg = bp->d_seg;
    a.chunk = bp->d_chunk;
    a.piece = bp->d_piece;
    a.deps = bp->d_deps;
    a.expect = bp->d_expect;
    a.cnt = bp->d_cnt;
    a.nseg = (int)bp->fo.seg.size();
    a.nreg = bp->fo.nreg;
    H2_CUDA_TRY(launch_seg<true>(a, rt, ops[0]->nsm, smem, s, &bp->grid));
    return H2_OK;
}

}  // namespace h2

// ---------------------------------------------------------------------------
// h2_matvec_noalloc: the same product with a fixed, library-owned workspace.
//
// Some callers cannot allocate device memory when they apply the operator:
// a time-stepping loop that reserved all of its device memory up front, an
// application whose memory belongs to its own pool allocator, or code that
// must not pay the device-wide synchronisation that cudaMalloc/cudaFree can
// cause.  For them this variant takes its workspace (the permuted input and
// the per-cluster x-hat / y-hat vectors) from the file-scope array below
// instead of from the operator's own allocation.  It calls no allocating
// CUDA or library routine.  It runs the level-wise schedule.
//
// The array is H2_STATIC_WS_DOUBLES doubles (32 MiB) on every GPU that loads
// this library, held until the process exits.  In host code its name is a
// host-side stand-in, not a device address: the device address is obtained
// once per device with cudaGetSymbolAddress (with that device current) on the
// first call, which also makes the runtime load this module on that device.
// Make that first call before any stream capture.  All calls share the one
// array and it keeps the last call's contents; the gather kernel rewrites the
// input rows and clears the accumulated y-hat rows on every call.  Calls whose
// executions overlap on the GPU (different streams, different operators)
// race on the array and give wrong results: serialise them.
// ---------------------------------------------------------------------------
#define H2_STATIC_WS_DOUBLES ((size_t)1 << 22)
static __device__ __align__(256) double g_h2_static_ws[H2_STATIC_WS_DOUBLES];

namespace h2 {
namespace {
constexpr int kMaxDevices = 64;
double* g_static_ws_dev[kMaxDevices] = {nullptr};
std::mutex g_static_ws_mu;

int static_workspace(double** out) {
    int dev = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return H2_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_static_ws_mu);
    if (!g_static_ws_dev[dev]) {
        void* p = nullptr;
        H2_CUDA_TRY(cudaGetSymbolAddress(&p, g_h2_static_ws));
        g_static_ws_dev[dev] = static_cast<double*>(p);
    }
    *out = g_static_ws_dev[dev];
    return H2_OK;
}

bool device_pointer(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
}  // namespace
}  // namespace h2

extern "C" int h2_matvec_noalloc(h2_handle* op, const double* u1, double* u2, int32_t r,
                                 void* cuda_stream) {
    using namespace h2;
    if (!op || !u1 || !u2) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    if (r < 1) return H2_ERR_INVALID_ARG;
    // a stage holds every chunk's inputs: operators built for at most 8
    // right-hand sides (128-column chunks) take r <= 8, the others r <= 32
    if (r > H2_MAX_RHS || (int64_t)op->chunk_cols * r > (int64_t)xin_cols(rt_for(r)) * rt_for(r)) {
        set_last_error(op->chunk_cols > xin_cols(H2_MAX_RHS)
                           ? "h2_matvec_noalloc: r > 8 needs an operator assembled with max_rhs > 8"
                           : "h2_matvec_noalloc: r > 32");
        return H2_ERR_RHS_EXCEEDS_MAX;
    }
    int dev = -1;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != op->device) {
        set_last_error("h2_matvec_noalloc: the current device is not the operator's device");
        return H2_ERR_INVALID_ARG;
    }
    const int64_t N = op->geom->N;
    const size_t bytes = sizeof(double) * (size_t)N * r;
    const char *a = (const char*)u1, *b = (const char*)u2;
    if (a < b + bytes && b < a + bytes) return H2_ERR_INVALID_ARG;
    if (!device_pointer(u1) || !device_pointer(u2)) return H2_ERR_INVALID_ARG;
    // FP64 workspace, then (FP32 operators) the FP32 workspace at a 256-byte boundary
    const size_t n64 = (size_t)op->ws_rows * (size_t)r;
    const size_t off32 = (n64 + 31) / 32 * 32;
    const size_t need = op->params.precision != H2_FP64 ? off32 + (n64 + 1) / 2 : n64;
    if (need > H2_STATIC_WS_DOUBLES) {
        set_last_error("h2_matvec_noalloc: the workspace of this operator and r exceeds the fixed 32 MiB scratch");
        return H2_ERR_SCRATCH_LIMIT;
    }
    double* ws = nullptr;
    int rc = static_workspace(&ws);
    if (rc != H2_OK) return rc;
    float* ws32 = op->params.precision != H2_FP64 ? reinterpret_cast<float*>(ws + off32) : nullptr;
    return launch_matvec(op, u1, u2, r, (cudaStream_t)cuda_stream, ws, ws32, false, nullptr, nullptr);
}
