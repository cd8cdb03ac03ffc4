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
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
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
    int32_t piece0, npieces;
    int32_t out_row, nrows, mode, signal;
};

struct KArgs {
    const FlowSeg* seg;        // segments (dataflow form: in ticket order)
    const Chunk* chunk;
    const Piece* piece;
    const int32_t* deps;       // dataflow form only
    const int32_t* expect;     // dataflow form only
    int32_t* cnt;              // dataflow form: region counters, ticket counter at [nreg]
    const unsigned char* arena;
    double* ws;
    double* u2;
    const int32_t* perm;
    int* err;
    int64_t N;
    int nseg;
    int nreg;
    int r;
    int stages;
    int stage_bytes;
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
__device__ __forceinline__ void signal_region(int32_t* p) {
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(p) : "memory");
}

// The producer warp's cursor over the chunks of its CTA (lane 0).
// FLOW: segments come from the global ticket counter (topological order);
// otherwise segments blockIdx.x, blockIdx.x + gridDim.x, ... of one pass.
template <bool FLOW>
struct Cursor {
    int seg = -1, ci = 0, nchunks = 0, k = 0, done = 0;
    __device__ void next(const KArgs& a, int& out_seg, int& out_ci) {
        out_seg = -1;
        out_ci = 0;
        while (!done) {
            if (seg >= 0 && ci < nchunks) {
                out_seg = seg;
                out_ci = ci++;
                return;
            }
            int t;
            if (FLOW) t = atomicAdd(a.cnt + a.nreg, 1);
            else t = (int)blockIdx.x + (k++) * (int)gridDim.x;
            if (t >= a.nseg) {
                done = 1;
                return;
            }
            seg = t;
            ci = 0;
            nchunks = a.seg[t].s.nchunks;
        }
    }
};

// Bounded wait (lane 0 of the producer) until every region segment `sg`
// reads has all its producers done.  False on timeout or abort.
__device__ bool deps_wait(const KArgs& a, int sg, volatile int* abort_flag) {
    const FlowSeg& F = a.seg[sg];
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

// The producer warp copies the input values of chunk C (the workspace rows of
// its pieces, concatenated, r values per row) into a stage's input buffer
// laid out [column of the chunk][RT], FP64 or (FP32 chunks) FP32.  Inputs are
// read through L2 (ld.global.cg): in the dataflow form other CTAs of the same
// launch wrote them.
template <int RT>
__device__ __forceinline__ void stage_inputs(const KArgs& a, const Chunk& C, unsigned char* xin, int lane) {
    constexpr int B = 8;   // loads in flight per lane
    const int r = a.r;
    const int total = C.ncols * r;
    const bool f32 = a.piece[C.piece0].type == PIECE_F32;
    int p = C.piece0, col0 = 0;
    Piece P = a.piece[p];
    for (int base = 0; base < total; base += 32 * B) {
        double v[B];
        int dst[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int idx = base + lane + 32 * j;
            dst[j] = -1;
            if (idx < total) {
                const int col = idx / r, cc = idx - col * r;
                while (col >= col0 + P.ncols) {
                    col0 += P.ncols;
                    P = a.piece[++p];
                }
                v[j] = __ldcg(a.ws + (int64_t)(P.in_row + col - col0) * r + cc);
                dst[j] = col * RT + cc;
            }
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
            if (dst[j] < 0) continue;
            if (f32) reinterpret_cast<float*>(xin)[dst[j]] = (float)v[j];
            else reinterpret_cast<double*>(xin)[dst[j]] = v[j];
        }
    }
}

// Multiplies the pieces of one staged chunk into the thread's accumulators.
template <int RT>
__device__ __forceinline__ void consume_chunk(const unsigned char* stage, int piece0, int npieces,
                                              const Piece* __restrict__ pieces, const unsigned char* xin,
                                              int r, int nrows, int row, int g, int G, double (&acc)[RT]) {
    int xcol = 0;
    for (int p = piece0; p < piece0 + npieces; ++p) {
        const Piece P = pieces[p];
        const int nc = P.ncols;
        if (P.type == PIECE_F64) {
            const double* A = reinterpret_cast<const double*>(stage + P.smem_off) + row;
            const double* x = reinterpret_cast<const double*>(xin) + xcol * RT;
            if (RT == 1) {
                double a0 = 0.0, a1 = 0.0;
                int col = g;
#pragma unroll 4
                for (; col + G < nc; col += 2 * G) {
                    a0 = fma(A[col * nrows], x[col], a0);
                    a1 = fma(A[(col + G) * nrows], x[col + G], a1);
                }
                if (col < nc) a0 = fma(A[col * nrows], x[col], a0);
                acc[0] += a0 + a1;
            } else {
#pragma unroll 2
                for (int col = g; col < nc; col += G) {
                    const double v = A[col * nrows];
#pragma unroll
                    for (int c = 0; c < RT; ++c)
                        if (c < r) acc[c] = fma(v, x[col * RT + c], acc[c]);
                }
            }
        } else {
            const float* A = reinterpret_cast<const float*>(stage + P.smem_off) + row;
            const float* x = reinterpret_cast<const float*>(xin) + xcol * RT;
            if (RT == 1) {
                float a0 = 0.0f, a1 = 0.0f;
                int col = g;
#pragma unroll 4
                for (; col + G < nc; col += 2 * G) {
                    a0 = fmaf(A[col * nrows], x[col], a0);
                    a1 = fmaf(A[(col + G) * nrows], x[col + G], a1);
                }
                if (col < nc) a0 = fmaf(A[col * nrows], x[col], a0);
                acc[0] += (double)(a0 + a1);
            } else {
                float acc32[RT];
#pragma unroll
                for (int c = 0; c < RT; ++c) acc32[c] = 0.0f;
#pragma unroll 2
                for (int col = g; col < nc; col += G) {
                    const float v = A[col * nrows];
#pragma unroll
                    for (int c = 0; c < RT; ++c)
                        if (c < r) acc32[c] = fmaf(v, x[col * RT + c], acc32[c]);
                }
#pragma unroll
                for (int c = 0; c < RT; ++c) acc[c] += (double)acc32[c];
            }
        }
        xcol += nc;
    }
}

// Adds the G partial sums of every row and writes the segment (consumer threads).
template <int RT>
__device__ __forceinline__ void write_segment(const StageDesc& D, const double* red, int r, int G,
                                              double* ws, double* u2, const int32_t* __restrict__ perm,
                                              int64_t N) {
    const int nrows = D.nrows;
    for (int idx = threadIdx.x; idx < nrows * r; idx += kConsumers) {
        const int rr = idx / r, c = idx - rr * r;
        double s = 0.0;
        for (int g2 = 0; g2 < G; ++g2) s += red[(g2 * nrows + rr) * RT + c];
        if (D.mode == SEG_FINAL || D.mode == SEG_FINAL_ADD) {
            double* dst = u2 + (int64_t)c * N + perm[D.out_row + rr];
            if (D.mode == SEG_FINAL) *dst = s;
            else *dst = __ldcg(dst) + s;
        } else {
            double* dst = ws + (int64_t)(D.out_row + rr) * r + c;
            if (D.mode == SEG_STORE) *dst = s;
            else if (D.mode == SEG_ADD) *dst = __ldcg(dst) + s;
            else atomicAdd(dst, s);
        }
    }
}

// Shared-memory layout of the segment kernel (dynamic part):
//   stages x stage_bytes             matrix chunks (bulk copies)
//   stages x kMaxChunkCols*RT*8      the chunks' input values
//   kConsumers * RT doubles          partial sums of the row groups
//   stages x 2 + 1 mbarriers         full[], empty[], segment barrier
//
// Warp specialisation.  The producer warp (the last warp) walks this CTA's
// chunks: it waits until the consumers released the stage, issues the bulk
// copy of the chunk's matrices, waits (dataflow form, first chunk of a
// segment, bounded) until the regions the segment reads are complete, copies
// the chunk's input values into the stage, publishes a descriptor and
// arrives on the stage's `full` barrier, which completes when the copy has
// landed.  The 8 consumer warps wait on `full`, multiply, release the stage
// on `empty` and, at the end of a segment, reduce and write it (and signal
// its region), synchronising among themselves on an mbarrier.  No CTA-wide
// barrier is taken per chunk and no wait is unbounded.
template <int RT, bool FLOW>
__global__ void __launch_bounds__(kBlock, 1) k_seg(const KArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = a.stages;
    constexpr size_t kXin = sizeof(double) * kMaxChunkCols * RT;
    unsigned char* stage_base = smem;
    unsigned char* xbase = smem + (size_t)S * a.stage_bytes;
    double* red = reinterpret_cast<double*>(xbase + (size_t)S * kXin);
    uint64_t* full = reinterpret_cast<uint64_t*>(red + kConsumers * RT);
    uint64_t* empty = full + S;
    uint64_t* segbar = empty + S;
    __shared__ StageDesc sd[kMaxStages];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 2);
            mbar_init(&empty[s], kConsumers);
        }
        mbar_init(segbar, kConsumers);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    volatile int* abortp = &abort_flag;
    int issued = 0;   // producer: chunks whose copy was issued

    if (tid >= kConsumers) {
        // ---------------- producer warp ----------------
        const int lane = tid & 31;
        Cursor<FLOW> cur;
        for (int i = 0;; ++i) {
            const int st = i % S;
            if (i >= S) {
                bool ok = true;
                if (lane == 0) ok = mbar_wait_or_abort(&empty[st], (uint32_t)((i / S) - 1) & 1u, abortp);
                if (!__shfl_sync(~0u, ok, 0)) break;
            }
            int sg = -1, ci = 0;
            if (lane == 0) cur.next(a, sg, ci);
            sg = __shfl_sync(~0u, sg, 0);
            ci = __shfl_sync(~0u, ci, 0);
            if (sg < 0) {   // end marker: complete the phase without a copy
                if (lane == 0) {
                    sd[st].seg = -1;
                    mbar_arrive(&full[st]);
                    mbar_arrive(&full[st]);
                }
                break;
            }
            const FlowSeg F = a.seg[sg];
            const Chunk C = a.chunk[F.s.chunk0 + ci];
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load(stage_base + (size_t)st * a.stage_bytes, a.arena + C.src, (uint32_t)C.bytes, &full[st]);
            }
            ++issued;
            bool ok = true;
            if (FLOW && ci == 0 && lane == 0) ok = deps_wait(a, sg, abortp);
            if (!__shfl_sync(~0u, ok, 0)) {
                if (lane == 0) {
                    atomicExch(a.err, 1);
                    abort_flag = 1;
                    sd[st].seg = -1;
                    mbar_arrive(&full[st]);
                }
                break;
            }
            stage_inputs<RT>(a, C, xbase + (size_t)st * kXin, lane);
            __syncwarp();
            if (lane == 0) {
                StageDesc D;
                D.seg = sg;
                D.last = ci == F.s.nchunks - 1;
                D.piece0 = C.piece0;
                D.npieces = C.npieces;
                D.out_row = F.s.out_row;
                D.nrows = F.s.nrows;
                D.mode = F.s.mode;
                D.signal = F.signal;
                sd[st] = D;
                mbar_arrive(&full[st]);
            }
        }
    } else {
        // ---------------- consumer warps ----------------
        const int r = a.r;
        double acc[RT];
#pragma unroll
        for (int c = 0; c < RT; ++c) acc[c] = 0.0;
        uint32_t segphase = 0;
        for (int i = 0;; ++i) {
            const int st = i % S;
            if (!mbar_wait_or_abort(&full[st], (uint32_t)(i / S) & 1u, abortp)) {
                atomicExch(a.err, 1);
                abort_flag = 1;
                break;
            }
            const StageDesc D = sd[st];
            if (D.seg < 0) break;
            const int nrows = D.nrows;
            const int G = kConsumers / nrows;
            const int row = tid % nrows, g = tid / nrows;
            if (g < G)
                consume_chunk<RT>(stage_base + (size_t)st * a.stage_bytes, D.piece0, D.npieces, a.piece,
                                  xbase + (size_t)st * kXin, r, nrows, row, g, G, acc);
            mbar_arrive(&empty[st]);
            if (D.last) {
                if (g < G) {
#pragma unroll
                    for (int c = 0; c < RT; ++c) red[tid * RT + c] = acc[c];
                }
#pragma unroll
                for (int c = 0; c < RT; ++c) acc[c] = 0.0;
                mbar_arrive(segbar);
                if (!mbar_wait_or_abort(segbar, segphase++ & 1u, abortp)) {
                    atomicExch(a.err, 1);
                    abort_flag = 1;
                    break;
                }
                write_segment<RT>(D, red, r, G, a.ws, a.u2, a.perm, a.N);
                if (FLOW) __threadfence();
                mbar_arrive(segbar);
                if (!mbar_wait_or_abort(segbar, segphase++ & 1u, abortp)) {
                    atomicExch(a.err, 1);
                    abort_flag = 1;
                    break;
                }
                if (FLOW && tid == 0 && D.signal >= 0) signal_region(a.cnt + D.signal);
            }
        }
    }
    __syncthreads();
    // after an abort, let the producer's copies still in flight land (bounded)
    if (tid == kConsumers && abort_flag) {
        for (int j = issued > S ? issued - S : 0; j < issued; ++j)
            (void)mbar_wait(&full[j % S], (uint32_t)(j / S) & 1u);
    }
}

// Gathers the input into tree order (workspace rows [0, N)), clears the
// y-hat rows that are accumulated atomically, and clears `nclear` ints (the
// flow kernel's region and ticket counters).
__global__ void k_prologue(const double* __restrict__ u1, double* __restrict__ ws,
                           const int32_t* __restrict__ perm, int64_t N, int r,
                           const int32_t* __restrict__ zero_rows, int nzero, int kp,
                           int32_t* __restrict__ clear, int nclear) {
    const int64_t tot = N * r;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t idx = i0; idx < tot; idx += stride) {
        const int64_t q = idx / r, c = idx - q * r;
        ws[idx] = u1[c * N + perm[q]];
    }
    const int64_t per = (int64_t)kp * r;
    const int64_t totz = (int64_t)nzero * per;
    for (int64_t idx = i0; idx < totz; idx += stride) {
        const int64_t z = idx / per, j = idx - z * per;
        ws[(int64_t)zero_rows[z] * r + j] = 0.0;
    }
    for (int64_t idx = i0; idx < nclear; idx += stride) clear[idx] = 0;
}

// Shared-memory stages of the segment kernel for r <= rt right-hand sides.
int stages_for(int rt) { return rt >= 32 ? 2 : 3; }

int rt_for(int r) {
    int rt = 1;
    while (rt < r) rt *= 2;
    return rt;
}

// Allows `smem` bytes of dynamic shared memory and asks for the largest
// shared-memory carveout, so that as many CTAs as fit are resident per SM.
template <class F>
cudaError_t set_smem(F* kernel, size_t smem, size_t& configured) {
    if (configured >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) configured = smem;
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
template <int RT, bool FLOW>
cudaError_t launch_seg_rt(const KArgs& a, int nsm, size_t smem, cudaStream_t s, int* launched) {
    static size_t configured = 0, occ_smem = 0;
    static int occ = 0;
    cudaError_t e = set_smem(k_seg<RT, FLOW>, smem, configured);
    if (e != cudaSuccess) return e;
    const int g = std::max(1, std::min(a.nseg, nsm * ctas_per_sm(k_seg<RT, FLOW>, smem, occ, occ_smem)));
    if (launched) *launched = g;
    k_seg<RT, FLOW><<<g, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

template <int RT>
int seg_occupancy(size_t smem) {
    static size_t configured = 0;
    if (set_smem(k_seg<RT, true>, smem, configured) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_seg<RT, true>, kBlock, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    return n;
}

template <bool FLOW>
cudaError_t launch_seg(const KArgs& a, int rt, int nsm, size_t smem, cudaStream_t s, int* launched) {
    switch (rt) {
        case 1: return launch_seg_rt<1, FLOW>(a, nsm, smem, s, launched);
        case 2: return launch_seg_rt<2, FLOW>(a, nsm, smem, s, launched);
        case 4: return launch_seg_rt<4, FLOW>(a, nsm, smem, s, launched);
        case 8: return launch_seg_rt<8, FLOW>(a, nsm, smem, s, launched);
        case 16: return launch_seg_rt<16, FLOW>(a, nsm, smem, s, launched);
        default: return launch_seg_rt<32, FLOW>(a, nsm, smem, s, launched);
    }
}

template <class T>
int upload_vec(const std::vector<T>& v, T** d) {
    H2_CUDA_TRY(cudaMalloc((void**)d, sizeof(T) * std::max<size_t>(1, v.size())));
    if (!v.empty()) H2_CUDA_TRY(cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return H2_OK;
}

// Launches the gather kernel and every pass (level-wise) or the flow kernel
// on workspace `ws`.
int launch_matvec(h2_handle* op, const double* u1, double* u2, int r, cudaStream_t s, double* ws,
                  bool flow, std::vector<cudaEvent_t>* marks,
                  std::vector<cudaEvent_t>* pool) {
    const int rt = rt_for(r);
    const size_t smem = pass_smem_bytes(op, rt);
    const int64_t N = op->geom->N;
    auto mark = [&]() -> cudaError_t {
        if (!marks) return cudaSuccess;
        cudaEvent_t e;
        if (!pool->empty()) {
            e = pool->back();
            pool->pop_back();
        } else {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
        }
        marks->push_back(e);
        return cudaEventRecord(e, s);
    };
    H2_CUDA_TRY(mark());
    {
        const std::vector<int32_t>& zr = flow ? op->fzero_rows : op->zero_rows;
        const int32_t* d_zr = flow ? op->d_fzero_rows : op->d_zero_rows;
        const int nclear = flow ? 3 * op->nc + 1 : 0;
        const int64_t work = std::max<int64_t>({N * r, (int64_t)zr.size() * op->kp * r, (int64_t)nclear});
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096));
        k_prologue<<<grid, 256, 0, s>>>(u1, ws, op->d_perm, N, r, d_zr, (int)zr.size(), op->kp,
                                        op->d_fcnt, nclear);
        H2_CUDA_TRY(cudaGetLastError());
    }
    H2_CUDA_TRY(mark());
    KArgs a{};
    a.arena = op->d_arena;
    a.ws = ws;
    a.u2 = u2;
    a.perm = op->d_perm;
    a.err = op->d_err;
    a.N = N;
    a.r = r;
    a.stages = stages_for(rt);
    a.stage_bytes = op->stage_bytes;
    if (flow) {
        a.seg = op->d_fseg;
        a.chunk = op->d_fchunk;
        a.piece = op->d_fpiece;
        a.deps = op->d_fdeps;
        a.expect = op->d_fexpect;
        a.cnt = op->d_fcnt;
        a.nseg = (int)op->fseg.size();
        a.nreg = 3 * op->nc;
        H2_CUDA_TRY(launch_seg<true>(a, rt, op->nsm, smem, s, &op->flow_grid));
        H2_CUDA_TRY(mark());
        return H2_OK;
    }
    for (Pass& p : op->passes) {
        a.seg = p.d_seg;
        a.chunk = p.d_chunk;
        a.piece = p.d_piece;
        a.nseg = (int)p.seg.size();
        H2_CUDA_TRY(launch_seg<false>(a, rt, op->nsm, smem, s, &p.grid));
        H2_CUDA_TRY(mark());
    }
    return H2_OK;
}

}  // namespace

size_t pass_smem_bytes(const h2_handle* op, int rt) {
    const size_t S = (size_t)stages_for(rt);
    return S * op->stage_bytes + S * sizeof(double) * kMaxChunkCols * rt + sizeof(double) * kConsumers * rt +
           sizeof(uint64_t) * (2 * S + 1);
}

// Resident CTAs and per-CTA rates of the dataflow kernel on the current
// device for the operator's largest r (input of the ticket-order simulation).
int flow_model(h2_handle* op, FlowModel& fm) {
    int dev = 0, nsm = 0, khz = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    H2_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    H2_CUDA_TRY(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    const int rt = rt_for(op->params.max_rhs);
    const size_t smem = pass_smem_bytes(op, rt);
    int occ = 1;
    switch (rt) {
        case 1: occ = seg_occupancy<1>(smem); break;
        case 2: occ = seg_occupancy<2>(smem); break;
        case 4: occ = seg_occupancy<4>(smem); break;
        case 8: occ = seg_occupancy<8>(smem); break;
        case 16: occ = seg_occupancy<16>(smem); break;
        default: occ = seg_occupancy<32>(smem); break;
    }
    const double ghz = khz > 0 ? khz * 1e-6 : 2.07;
    fm.workers = nsm * occ;
    fm.r = op->params.max_rhs;
    fm.f64_per_ns = 2.0 * ghz / occ;
    fm.f32_per_ns = 128.0 * ghz / occ;
    fm.bytes_per_ns = 6800.0 / fm.workers;
    return H2_OK;
}

int upload_plan(h2_handle* op) {
    int dev = 0, nsm = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    H2_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int rc;
    for (Pass& p : op->passes) {
        std::vector<FlowSeg> fs(p.seg.size());
        for (size_t i = 0; i < p.seg.size(); ++i) fs[i] = FlowSeg{p.seg[i], -1, 0, 0, p.kind};
        if ((rc = upload_vec(fs, &p.d_seg)) || (rc = upload_vec(p.chunk, &p.d_chunk)) ||
            (rc = upload_vec(p.piece, &p.d_piece)))
            return rc;
        p.grid = 0;
    }
    op->nsm = nsm;
    if ((rc = upload_vec(op->zero_rows, &op->d_zero_rows))) return rc;
    if (op->use_flow) {
        if ((rc = upload_vec(op->fseg, &op->d_fseg)) || (rc = upload_vec(op->fchunk, &op->d_fchunk)) ||
            (rc = upload_vec(op->fpiece, &op->d_fpiece)) || (rc = upload_vec(op->fdeps, &op->d_fdeps)) ||
            (rc = upload_vec(op->fexpect, &op->d_fexpect)) ||
            (rc = upload_vec(op->fzero_rows, &op->d_fzero_rows)))
            return rc;
        H2_CUDA_TRY(cudaMalloc((void**)&op->d_fcnt, sizeof(int32_t) * (3 * (size_t)op->nc + 1)));
    }
    H2_CUDA_TRY(cudaMalloc((void**)&op->d_ws, sizeof(double) * (size_t)op->ws_rows * op->params.max_rhs));
    H2_CUDA_TRY(cudaMalloc((void**)&op->d_err, sizeof(int)));
    H2_CUDA_TRY(cudaMemset(op->d_err, 0, sizeof(int)));
    op->n_launches = op->use_flow ? 2 : 1 + (int)op->passes.size();
    return H2_OK;
}

void release_graph(h2_handle* op) {
    if (op->graph_exec) cudaGraphExecDestroy(op->graph_exec);
    if (op->graph) cudaGraphDestroy(op->graph);
    op->graph_exec = nullptr;
    op->graph = nullptr;
    op->graph_r = 0;
}

void release_profile(h2_handle* op) {
    for (auto& call : op->prof_calls)
        for (cudaEvent_t e : call) cudaEventDestroy(e);
    for (cudaEvent_t e : op->prof_pool) cudaEventDestroy(e);
    op->prof_calls.clear();
    op->prof_pool.clear();
}

int read_profile(h2_handle* op, std::vector<double>& ms, int& ncalls) {
    ms.clear();
    ncalls = (int)op->prof_calls.size();
    for (auto& call : op->prof_calls) {
        H2_CUDA_TRY(cudaEventSynchronize(call.back()));
        if (ms.size() < call.size() - 1) ms.resize(call.size() - 1, 0.0);
        for (size_t i = 0; i + 1 < call.size(); ++i) {
            float t = 0.0f;
            H2_CUDA_TRY(cudaEventElapsedTime(&t, call[i], call[i + 1]));
            ms[i] += t;
        }
        for (cudaEvent_t e : call) op->prof_pool.push_back(e);
    }
    op->prof_calls.clear();
    return H2_OK;
}

int matvec_device(h2_handle* op, const double* u1, double* u2, int r, cudaStream_t s) {
    std::vector<cudaEvent_t> ev;
    int rc = launch_matvec(op, u1, u2, r, s, op->d_ws, op->use_flow != 0,
                           op->prof_enabled ? &ev : nullptr, &op->prof_pool);
    if (op->prof_enabled) op->prof_calls.push_back(std::move(ev));
    return rc;
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
    if (r < 1 || r > H2_MAX_RHS) return H2_ERR_INVALID_ARG;
    const int64_t N = op->geom->N;
    const size_t bytes = sizeof(double) * (size_t)N * r;
    const char *a = (const char*)u1, *b = (const char*)u2;
    if (a < b + bytes && b < a + bytes) return H2_ERR_INVALID_ARG;
    if (!device_pointer(u1) || !device_pointer(u2)) return H2_ERR_INVALID_ARG;
    if ((size_t)op->ws_rows * (size_t)r > H2_STATIC_WS_DOUBLES) {
        set_last_error("h2_matvec_noalloc: workspace rows x r exceeds the fixed scratch of 4194304 doubles");
        return H2_ERR_SCRATCH_LIMIT;
    }
    double* ws = nullptr;
    int rc = static_workspace(&ws);
    if (rc != H2_OK) return rc;
    return launch_matvec(op, u1, u2, r, (cudaStream_t)cuda_stream, ws, false, nullptr, nullptr);
}

#ifdef H2_TRACE
// Copies the first n segment records of the last traced flow launch to host.
extern "C" int h2_trace_read(long long* out, int n) {
    if (cudaDeviceSynchronize() != cudaSuccess) return H2_ERR_CUDA;
    if (cudaMemcpyFromSymbol(out, h2::g_h2_trace, sizeof(long long) * 5 * (size_t)n) != cudaSuccess)
        return H2_ERR_CUDA;
    return H2_OK;
}
#endif
