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

constexpr int kThreads = 256;
constexpr int kQueue = 16;                               // segment queue of the flow kernel
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

// Copies the input slices of the pieces of one chunk into shared memory
// (FP64, or FP32 for FP32 pieces): one L2 read per value instead of one per
// thread and column.  Inputs are read through L2 (ld.global.cg): in the flow
// kernel they are written by other CTAs of the same launch.
template <int RT>
__device__ __forceinline__ void stage_inputs(const Chunk& C, const Piece* __restrict__ pieces,
                                             const double* __restrict__ ws, int r, unsigned char* xin) {
    int off = 0;   // bytes
    for (int p = C.piece0; p < C.piece0 + C.npieces; ++p) {
        const Piece P = pieces[p];
        const double* __restrict__ in = ws + (int64_t)P.in_row * r;
        const int n = P.ncols * r;
        if (P.type == PIECE_F64) {
            double* x = reinterpret_cast<double*>(xin + off);
            for (int idx = threadIdx.x; idx < n; idx += kThreads) {
                const int j = idx / r, c = idx - j * r;
                x[j * RT + c] = __ldcg(in + idx);
            }
            off += P.ncols * RT * 8;
        } else {
            float* x = reinterpret_cast<float*>(xin + off);
            for (int idx = threadIdx.x; idx < n; idx += kThreads) {
                const int j = idx / r, c = idx - j * r;
                x[j * RT + c] = (float)__ldcg(in + idx);
            }
            off += ((P.ncols * RT * 4 + 15) & ~15);
        }
    }
}

// Multiplies the pieces of one staged chunk into the thread's accumulators.
template <int RT>
__device__ __forceinline__ void consume_chunk(const unsigned char* stage, const Chunk& C,
                                              const Piece* __restrict__ pieces, const unsigned char* xin,
                                              int r, int nrows, int row, int g, int G, double (&acc)[RT]) {
    int off = 0;
    for (int p = C.piece0; p < C.piece0 + C.npieces; ++p) {
        const Piece P = pieces[p];
        const int nc = P.ncols;
        if (P.type == PIECE_F64) {
            const double* A = reinterpret_cast<const double*>(stage + P.smem_off) + row;
            const double* x = reinterpret_cast<const double*>(xin + off);
            off += nc * RT * 8;
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
            const float* x = reinterpret_cast<const float*>(xin + off);
            off += ((nc * RT * 4 + 15) & ~15);
            if (RT == 1) {
                float a0 = 0.0f, a1 = 0.0f;
                int col = g;
#pragma unroll 4
                for (; col + G < nc; col += 2 * G) {
                    a0 = fmaf(A[col * nrows], x[col], a0);
                    a1 = fmaf(A[(col + G) * nrows], x[col + G], a1);
                }
                if (col < nc) a0 = fmaf(A[col * nrows], x[col], a0);
                acc[0] += (double)a0 + (double)a1;
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
    }
}

// Adds the G partial sums of every row and writes the segment.
template <int RT>
__device__ __forceinline__ void write_segment(const Segment& S, int mode, const double* red, int r,
                                              int G, double* ws, double* u2,
                                              const int32_t* __restrict__ perm, int64_t N) {
    const int nrows = S.nrows;
    for (int idx = threadIdx.x; idx < nrows * r; idx += kThreads) {
        const int rr = idx / r, c = idx - rr * r;
        double s = 0.0;
        for (int g2 = 0; g2 < G; ++g2) s += red[(g2 * nrows + rr) * RT + c];
        if (mode == SEG_FINAL || mode == SEG_FINAL_ADD) {
            double* dst = u2 + (int64_t)c * N + perm[S.out_row + rr];
            if (mode == SEG_FINAL) *dst = s;
            else *dst = __ldcg(dst) + s;
        } else {
            double* dst = ws + (int64_t)(S.out_row + rr) * r + c;
            if (mode == SEG_STORE) *dst = s;
            else if (mode == SEG_ADD) *dst = __ldcg(dst) + s;
            else atomicAdd(dst, s);
        }
    }
}

struct PassArgs {
    const Segment* seg;
    const Chunk* chunk;
    const Piece* piece;
    const unsigned char* arena;
    double* ws;
    double* u2;
    const int32_t* perm;
    int* err;
    int64_t N;
    int nseg;
    int r;
    int stages;
    int stage_bytes;
};

// Producer cursor over the chunks of the segments blockIdx.x, +gridDim.x, ...
struct Cursor {
    int seg, ci;
    __device__ int next(const PassArgs& a) {
        while (seg < a.nseg) {
            const Segment s = a.seg[seg];
            if (ci < s.nchunks) return s.chunk0 + ci++;
            seg += gridDim.x;
            ci = 0;
        }
        return -1;
    }
};

// One pass, segments assigned round-robin (the host sorts them longest first).
template <int RT>
__global__ void __launch_bounds__(kThreads, 1) k_pass(const PassArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage_base = smem;
    double* red = reinterpret_cast<double*>(smem + (size_t)a.stages * a.stage_bytes);
    unsigned char* xin = reinterpret_cast<unsigned char*>(red + kThreads * RT);
    uint64_t* full = reinterpret_cast<uint64_t*>(xin + (size_t)kMaxChunkCols * RT * 8);
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int r = a.r;
    Cursor prod{(int)blockIdx.x, 0};
    int issued = 0;   // chunks issued (thread 0)
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < a.stages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        for (int s = 0; s < a.stages; ++s) {
            const int c = prod.next(a);
            if (c < 0) break;
            const Chunk ch = a.chunk[c];
            tma_load(stage_base + (size_t)s * a.stage_bytes, a.arena + ch.src, (uint32_t)ch.bytes, &full[s]);
            ++issued;
        }
    }

    int it = 0;   // chunks consumed
    for (int sg = blockIdx.x; sg < a.nseg; sg += gridDim.x) {
        const Segment S = a.seg[sg];
        const int nrows = S.nrows;
        const int G = kThreads / nrows;
        const int row = tid % nrows, g = tid / nrows;
        const bool active = g < G;
        double acc[RT];
#pragma unroll
        for (int c = 0; c < RT; ++c) acc[c] = 0.0;

        for (int ci = 0; ci < S.nchunks; ++ci) {
            const int st = it % a.stages;
            const uint32_t parity = (uint32_t)(it / a.stages) & 1u;
            if (!mbar_wait(&full[st], parity)) abort_flag = 1;
            const Chunk C = a.chunk[S.chunk0 + ci];
            stage_inputs<RT>(C, a.piece, a.ws, r, xin);
            __syncthreads();   // staged inputs visible
            if (active)
                consume_chunk<RT>(stage_base + (size_t)st * a.stage_bytes, C, a.piece, xin, r, nrows,
                                  row, g, G, acc);
            __syncthreads();   // every thread is done with stage st
            if (abort_flag) goto bail;
            if (tid == 0) {
                const int c = prod.next(a);
                if (c >= 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    const Chunk ch = a.chunk[c];
                    tma_load(stage_base + (size_t)st * a.stage_bytes, a.arena + ch.src, (uint32_t)ch.bytes,
                             &full[st]);
                    ++issued;
                }
            }
            ++it;
        }
        if (active) {
#pragma unroll
            for (int c = 0; c < RT; ++c) red[tid * RT + c] = acc[c];
        }
        __syncthreads();
        write_segment<RT>(S, S.mode, red, r, G, a.ws, a.u2, a.perm, a.N);
        __syncthreads();
    }
    return;

bail:
    // a bulk copy did not complete in time: report it, let the copies still in
    // flight land (bounded), and leave
    if (tid == 0) {
        atomicExch(a.err, 1);
        for (int j = it; j < issued; ++j) {
            const int st = j % a.stages;
            (void)mbar_wait(&full[st], (uint32_t)(j / a.stages) & 1u);
        }
    }
    __syncthreads();
}

struct FlowArgs {
    const FlowSeg* seg;
    const Chunk* chunk;
    const Piece* piece;
    const int32_t* deps;
    const int32_t* expect;
    int32_t* cnt;            // region counters, then the ticket counter at [nreg]
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

// Producer side of the flow kernel (thread 0 only): hands out chunks of the
// segments this CTA took, taking a new ticket when a segment is exhausted.
struct FlowCursor {
    int seg, ci, qhead, done;
    __device__ int next(const FlowArgs& a, int* queue) {
        while (true) {
            if (seg >= 0 && ci < a.seg[seg].s.nchunks) return a.seg[seg].s.chunk0 + ci++;
            if (done) return -1;
            const int t = atomicAdd(a.cnt + a.nreg, 1);
            if (t >= a.nseg) {
                queue[qhead++ % kQueue] = -1;
                done = 1;
                return -1;
            }
            queue[qhead++ % kQueue] = t;
            seg = t;
            ci = 0;
        }
    }
};

#ifdef H2_TRACE
// Per-segment timeline (diagnostic builds only): ticket, SM, start, inputs
// ready, end (globaltimer ns).
__device__ long long g_h2_trace[1 << 22];
__device__ __forceinline__ unsigned smid() {
    unsigned v;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
    return v;
}
#endif

template <int RT>
__global__ void __launch_bounds__(kThreads, 1) k_flow(const FlowArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage_base = smem;
    double* red = reinterpret_cast<double*>(smem + (size_t)a.stages * a.stage_bytes);
    unsigned char* xin = reinterpret_cast<unsigned char*>(red + kThreads * RT);
    uint64_t* full = reinterpret_cast<uint64_t*>(xin + (size_t)kMaxChunkCols * RT * 8);
    __shared__ int queue[kQueue];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    const int r = a.r;
    FlowCursor prod{-1, 0, 0, 0};
    int issued = 0;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < a.stages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int s = 0; s < a.stages; ++s) {
            const int c = prod.next(a, queue);
            if (c < 0) break;
            const Chunk ch = a.chunk[c];
            tma_load(stage_base + (size_t)s * a.stage_bytes, a.arena + ch.src, (uint32_t)ch.bytes, &full[s]);
            ++issued;
        }
        if (issued == 0) queue[0] = -1;   // no work left for this CTA
    }

    int it = 0, qtail = 0;
    while (true) {
        __syncthreads();   // queue entry of the next segment is visible
        const int sg = queue[qtail++ % kQueue];
        if (sg < 0) break;
        const FlowSeg F = a.seg[sg];
        const Segment S = F.s;
#ifdef H2_TRACE
        long long tr0 = (long long)now_ns();
#endif
        // wait until every region this segment reads is complete
        if (tid == 0) {
            for (int d = F.dep0; d < F.dep0 + F.ndep && !abort_flag; ++d) {
                const int reg = a.deps[d];
                const int want = a.expect[reg];
                if (ld_acquire(a.cnt + reg) >= want) continue;
                const unsigned long long t0 = now_ns();
                while (ld_acquire(a.cnt + reg) < want) {
                    if (ld_acquire(a.err) != 0 || now_ns() - t0 > kWaitNs) {
                        abort_flag = 1;
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        __syncthreads();
        if (abort_flag) goto bail;
#ifdef H2_TRACE
        long long tr1 = (long long)now_ns();
#endif

        const int nrows = S.nrows;
        const int G = kThreads / nrows;
        const int row = tid % nrows, g = tid / nrows;
        const bool active = g < G;
        double acc[RT];
#pragma unroll
        for (int c = 0; c < RT; ++c) acc[c] = 0.0;
        for (int ci = 0; ci < S.nchunks; ++ci) {
            const int st = it % a.stages;
            const uint32_t parity = (uint32_t)(it / a.stages) & 1u;
            if (!mbar_wait(&full[st], parity)) abort_flag = 1;
            const Chunk C = a.chunk[S.chunk0 + ci];
            stage_inputs<RT>(C, a.piece, a.ws, r, xin);
            __syncthreads();   // staged inputs visible
            if (active)
                consume_chunk<RT>(stage_base + (size_t)st * a.stage_bytes, C, a.piece, xin, r, nrows,
                                  row, g, G, acc);
            __syncthreads();
            if (abort_flag) goto bail;
            if (tid == 0) {
                const int c = prod.next(a, queue);
                if (c >= 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    const Chunk ch = a.chunk[c];
                    tma_load(stage_base + (size_t)st * a.stage_bytes, a.arena + ch.src, (uint32_t)ch.bytes,
                             &full[st]);
                    ++issued;
                }
            }
            ++it;
        }
        if (active) {
#pragma unroll
            for (int c = 0; c < RT; ++c) red[tid * RT + c] = acc[c];
        }
        __syncthreads();
        write_segment<RT>(S, S.mode, red, r, G, a.ws, a.u2, a.perm, a.N);
        __threadfence();
        __syncthreads();
        if (tid == 0 && F.signal >= 0) atomicAdd(a.cnt + F.signal, 1);
#ifdef H2_TRACE
        if (tid == 0 && 5 * (sg + 1) < (1 << 22)) {
            long long* t = g_h2_trace + 5 * sg;
            t[0] = sg; t[1] = (long long)F.kind * 1000000 + smid() * 1000 + blockIdx.x % 1000; t[2] = tr0; t[3] = tr1;
            t[4] = (long long)now_ns();
        }
#endif
    }
    return;

bail:
    if (tid == 0) {
        atomicExch(a.err, 1);
        for (int j = it; j < issued; ++j) {
            const int st = j % a.stages;
            (void)mbar_wait(&full[st], (uint32_t)(j / a.stages) & 1u);
        }
    }
    __syncthreads();
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

int rt_for(int r) {
    int rt = 1;
    while (rt < r) rt *= 2;
    return rt;
}

template <class F>
cudaError_t set_smem(F* kernel, size_t smem, size_t& configured) {
    if (configured >= smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) configured = smem;
    return e;
}

// Resident CTAs per SM of a kernel at this shared-memory size (cached).
template <class F>
int ctas_per_sm(F* kernel, size_t smem, int& cached, size_t& cached_smem) {
    if (cached > 0 && cached_smem == smem) return cached;
    int n = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, smem) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = 1;
    }
    cached = n;
    cached_smem = smem;
    return n;
}

template <int RT>
cudaError_t launch_pass_rt(const PassArgs& a, int grid, size_t smem, cudaStream_t s) {
    static size_t configured = 0, occ_smem = 0;
    static int occ = 0;
    cudaError_t e = set_smem(k_pass<RT>, smem, configured);
    if (e != cudaSuccess) return e;
    const int g = std::max(1, std::min(a.nseg, grid * ctas_per_sm(k_pass<RT>, smem, occ, occ_smem)));
    k_pass<RT><<<g, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pass(const PassArgs& a, int rt, int grid, size_t smem, cudaStream_t s) {
    switch (rt) {
        case 1: return launch_pass_rt<1>(a, grid, smem, s);
        case 2: return launch_pass_rt<2>(a, grid, smem, s);
        case 4: return launch_pass_rt<4>(a, grid, smem, s);
        case 8: return launch_pass_rt<8>(a, grid, smem, s);
        case 16: return launch_pass_rt<16>(a, grid, smem, s);
        default: return launch_pass_rt<32>(a, grid, smem, s);
    }
}

template <int RT>
cudaError_t launch_flow_rt(const FlowArgs& a, int grid, size_t smem, cudaStream_t s) {
    static size_t configured = 0, occ_smem = 0;
    static int occ = 0;
    cudaError_t e = set_smem(k_flow<RT>, smem, configured);
    if (e != cudaSuccess) return e;
    const int g = std::max(1, std::min(a.nseg, grid * ctas_per_sm(k_flow<RT>, smem, occ, occ_smem)));
    k_flow<RT><<<g, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_flow(const FlowArgs& a, int rt, int grid, size_t smem, cudaStream_t s) {
    switch (rt) {
        case 1: return launch_flow_rt<1>(a, grid, smem, s);
        case 2: return launch_flow_rt<2>(a, grid, smem, s);
        case 4: return launch_flow_rt<4>(a, grid, smem, s);
        case 8: return launch_flow_rt<8>(a, grid, smem, s);
        case 16: return launch_flow_rt<16>(a, grid, smem, s);
        default: return launch_flow_rt<32>(a, grid, smem, s);
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
    if (flow) {
        FlowArgs a{};
        a.seg = op->d_fseg;
        a.chunk = op->d_fchunk;
        a.piece = op->d_fpiece;
        a.deps = op->d_fdeps;
        a.expect = op->d_fexpect;
        a.cnt = op->d_fcnt;
        a.arena = op->d_arena;
        a.ws = ws;
        a.u2 = u2;
        a.perm = op->d_perm;
        a.err = op->d_err;
        a.N = N;
        a.nseg = (int)op->fseg.size();
        a.nreg = 3 * op->nc;
        a.r = r;
        a.stages = op->stages;
        a.stage_bytes = op->stage_bytes;
        H2_CUDA_TRY(launch_flow(a, rt, op->flow_grid, smem, s));
        H2_CUDA_TRY(mark());
        return H2_OK;
    }
    for (const Pass& p : op->passes) {
        PassArgs a{};
        a.seg = p.d_seg;
        a.chunk = p.d_chunk;
        a.piece = p.d_piece;
        a.arena = op->d_arena;
        a.ws = ws;
        a.u2 = u2;
        a.perm = op->d_perm;
        a.err = op->d_err;
        a.N = N;
        a.nseg = (int)p.seg.size();
        a.r = r;
        a.stages = op->stages;
        a.stage_bytes = op->stage_bytes;
        H2_CUDA_TRY(launch_pass(a, rt, p.grid, smem, s));
        H2_CUDA_TRY(mark());
    }
    return H2_OK;
}

}  // namespace

size_t pass_smem_bytes(const h2_handle* op, int rt) {
    return (size_t)op->stages * op->stage_bytes + sizeof(double) * kThreads * rt +
           sizeof(double) * kMaxChunkCols * rt + sizeof(uint64_t) * op->stages;
}

int upload_plan(h2_handle* op) {
    int dev = 0, nsm = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    H2_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int rc;
    for (Pass& p : op->passes) {
        if ((rc = upload_vec(p.seg, &p.d_seg)) || (rc = upload_vec(p.chunk, &p.d_chunk)) ||
            (rc = upload_vec(p.piece, &p.d_piece)))
            return rc;
        p.grid = nsm;
    }
    if ((rc = upload_vec(op->zero_rows, &op->d_zero_rows))) return rc;
    if (op->use_flow) {
        if ((rc = upload_vec(op->fseg, &op->d_fseg)) || (rc = upload_vec(op->fchunk, &op->d_fchunk)) ||
            (rc = upload_vec(op->fpiece, &op->d_fpiece)) || (rc = upload_vec(op->fdeps, &op->d_fdeps)) ||
            (rc = upload_vec(op->fexpect, &op->d_fexpect)) ||
            (rc = upload_vec(op->fzero_rows, &op->d_fzero_rows)))
            return rc;
        H2_CUDA_TRY(cudaMalloc((void**)&op->d_fcnt, sizeof(int32_t) * (3 * (size_t)op->nc + 1)));
        op->flow_grid = nsm;
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
