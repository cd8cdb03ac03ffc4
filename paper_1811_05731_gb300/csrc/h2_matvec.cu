// The H2 matrix-vector product u2 = M u1 (arXiv:1811.05731, Eq. denseMat;
// Section "H2-Matrix Compression") on one GPU.
//
// One kernel, k_pass, executes every pass of the plan (upward leaf
// projection, upward transfers, coupling, downward transfers, leaf expansion
// with the near field).  A pass is a list of output segments; each segment
// sums column-major matrices times workspace vectors.  The matrices of a pass
// lie contiguously in HBM in the order the CTAs consume them and are streamed
// into a ring of shared-memory stages by one elected thread with bulk TMA
// copies (cp.async.bulk + mbarrier transaction counts).  The other threads
// compute from shared memory: thread (row, g) accumulates row `row` over the
// columns congruent to g modulo G, and the G partial sums are added in
// shared memory at the end of the segment.
//
// FP64 pieces accumulate in FP64.  FP32 pieces (far field of an FP32
// operator) multiply and accumulate in FP32 within one piece and add the
// piece's sum to the FP64 accumulator; the workspace and u2 are FP64.
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
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s bound on any mbarrier wait

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

template <int RT>
__global__ void __launch_bounds__(kThreads, 1) k_pass(const PassArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stage_base = smem;
    double* red = reinterpret_cast<double*>(smem + (size_t)a.stages * a.stage_bytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(red + kThreads * RT);
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
        const int R = (nrows + 31) & ~31;
        const int G = kThreads / R;
        const int row = tid % R, g = tid / R;
        const bool active = g < G && row < nrows;
        double acc[RT];
#pragma unroll
        for (int c = 0; c < RT; ++c) acc[c] = 0.0;

        for (int ci = 0; ci < S.nchunks; ++ci) {
            const int st = it % a.stages;
            const uint32_t parity = (uint32_t)(it / a.stages) & 1u;
            if (!mbar_wait(&full[st], parity)) abort_flag = 1;
            const Chunk C = a.chunk[S.chunk0 + ci];
            if (active) {
                for (int p = C.piece0; p < C.piece0 + C.npieces; ++p) {
                    const Piece P = a.piece[p];
                    const unsigned char* base = stage_base + (size_t)st * a.stage_bytes + P.smem_off;
                    const double* __restrict__ in = a.ws + (int64_t)P.in_row * r;
                    if (P.type == PIECE_F64) {
                        const double* A = reinterpret_cast<const double*>(base) + row;
#pragma unroll 4
                        for (int col = g; col < P.ncols; col += G) {
                            const double v = A[col * nrows];
                            if (RT == 1) {
                                acc[0] = fma(v, __ldg(in + col), acc[0]);
                            } else {
#pragma unroll
                                for (int c = 0; c < RT; ++c)
                                    if (c < r) acc[c] = fma(v, __ldg(in + (int64_t)col * r + c), acc[c]);
                            }
                        }
                    } else {
                        const float* A = reinterpret_cast<const float*>(base) + row;
                        float acc32[RT];
#pragma unroll
                        for (int c = 0; c < RT; ++c) acc32[c] = 0.0f;
#pragma unroll 4
                        for (int col = g; col < P.ncols; col += G) {
                            const float v = A[col * nrows];
                            if (RT == 1) {
                                acc32[0] = fmaf(v, (float)__ldg(in + col), acc32[0]);
                            } else {
#pragma unroll
                                for (int c = 0; c < RT; ++c)
                                    if (c < r)
                                        acc32[c] = fmaf(v, (float)__ldg(in + (int64_t)col * r + c), acc32[c]);
                            }
                        }
#pragma unroll
                        for (int c = 0; c < RT; ++c) acc[c] += (double)acc32[c];
                    }
                }
            }
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
        // combine the G partial sums of every row and write the segment
        if (active) {
#pragma unroll
            for (int c = 0; c < RT; ++c) red[tid * RT + c] = acc[c];
        }
        __syncthreads();
        for (int idx = tid; idx < nrows * r; idx += kThreads) {
            const int rr = idx / r, c = idx - rr * r;
            double s = 0.0;
            for (int g2 = 0; g2 < G; ++g2) s += red[(g2 * R + rr) * RT + c];
            if (S.mode == SEG_FINAL) {
                a.u2[(int64_t)c * a.N + a.perm[S.out_row + rr]] = s;
            } else {
                double* dst = a.ws + (int64_t)(S.out_row + rr) * r + c;
                if (S.mode == SEG_STORE) *dst = s;
                else if (S.mode == SEG_ADD) *dst += s;
                else atomicAdd(dst, s);
            }
        }
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

// Gathers the input into tree order (workspace rows [0, N)) and clears the
// y-hat rows that the coupling pass accumulates into.
__global__ void k_prologue(const double* __restrict__ u1, double* __restrict__ ws,
                           const int32_t* __restrict__ perm, int64_t N, int r,
                           const int32_t* __restrict__ zero_rows, int nzero, int kp) {
    const int64_t tot = N * r;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += stride) {
        const int64_t q = idx / r, c = idx - q * r;
        ws[idx] = u1[c * N + perm[q]];
    }
    const int64_t per = (int64_t)kp * r;
    const int64_t totz = (int64_t)nzero * per;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < totz; idx += stride) {
        const int64_t z = idx / per, j = idx - z * per;
        ws[(int64_t)zero_rows[z] * r + j] = 0.0;
    }
}

int rt_for(int r) {
    int rt = 1;
    while (rt < r) rt *= 2;
    return rt;
}

template <int RT>
cudaError_t launch_pass_rt(const PassArgs& a, int grid, size_t smem, cudaStream_t s) {
    static int configured = 0;
    static size_t configured_smem = 0;
    if (!configured || configured_smem < smem) {
        cudaError_t e = cudaFuncSetAttribute(k_pass<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = 1;
        configured_smem = smem;
    }
    k_pass<RT><<<grid, kThreads, smem, s>>>(a);
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

}  // namespace

size_t pass_smem_bytes(const h2_handle* op, int rt) {
    return (size_t)op->stages * op->stage_bytes + sizeof(double) * kThreads * rt +
           sizeof(uint64_t) * op->stages;
}

int upload_plan(h2_handle* op) {
    int dev = 0, nsm = 0;
    H2_CUDA_TRY(cudaGetDevice(&dev));
    H2_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    for (Pass& p : op->passes) {
        H2_CUDA_TRY(cudaMalloc((void**)&p.d_seg, sizeof(Segment) * std::max<size_t>(1, p.seg.size())));
        H2_CUDA_TRY(cudaMalloc((void**)&p.d_chunk, sizeof(Chunk) * std::max<size_t>(1, p.chunk.size())));
        H2_CUDA_TRY(cudaMalloc((void**)&p.d_piece, sizeof(Piece) * std::max<size_t>(1, p.piece.size())));
        H2_CUDA_TRY(cudaMemcpy(p.d_seg, p.seg.data(), sizeof(Segment) * p.seg.size(), cudaMemcpyHostToDevice));
        H2_CUDA_TRY(cudaMemcpy(p.d_chunk, p.chunk.data(), sizeof(Chunk) * p.chunk.size(), cudaMemcpyHostToDevice));
        H2_CUDA_TRY(cudaMemcpy(p.d_piece, p.piece.data(), sizeof(Piece) * p.piece.size(), cudaMemcpyHostToDevice));
        p.grid = (int)std::min<size_t>(p.seg.size(), (size_t)nsm);
    }
    if (!op->zero_rows.empty()) {
        H2_CUDA_TRY(cudaMalloc((void**)&op->d_zero_rows, sizeof(int32_t) * op->zero_rows.size()));
        H2_CUDA_TRY(cudaMemcpy(op->d_zero_rows, op->zero_rows.data(), sizeof(int32_t) * op->zero_rows.size(),
                               cudaMemcpyHostToDevice));
    }
    H2_CUDA_TRY(cudaMalloc((void**)&op->d_ws, sizeof(double) * (size_t)op->ws_rows * op->params.max_rhs));
    H2_CUDA_TRY(cudaMalloc((void**)&op->d_err, sizeof(int)));
    H2_CUDA_TRY(cudaMemset(op->d_err, 0, sizeof(int)));
    op->n_launches = 1 + (int)op->passes.size();
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
    ms.assign(op->passes.size() + 1, 0.0);
    ncalls = (int)op->prof_calls.size();
    for (auto& call : op->prof_calls) {
        H2_CUDA_TRY(cudaEventSynchronize(call.back()));
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
    const int rt = rt_for(r);
    const size_t smem = pass_smem_bytes(op, rt);
    const int64_t N = op->geom->N;
    std::vector<cudaEvent_t> ev;
    auto mark = [&]() -> cudaError_t {
        if (!op->prof_enabled) return cudaSuccess;
        cudaEvent_t e;
        if (!op->prof_pool.empty()) {
            e = op->prof_pool.back();
            op->prof_pool.pop_back();
        } else {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) return err;
        }
        ev.push_back(e);
        return cudaEventRecord(e, s);
    };
    H2_CUDA_TRY(mark());
    {
        const int64_t work = std::max<int64_t>(N * r, (int64_t)op->zero_rows.size() * op->kp * r);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096));
        k_prologue<<<grid, 256, 0, s>>>(u1, op->d_ws, op->d_perm, N, r, op->d_zero_rows,
                                        (int)op->zero_rows.size(), op->kp);
        H2_CUDA_TRY(cudaGetLastError());
    }
    H2_CUDA_TRY(mark());
    for (const Pass& p : op->passes) {
        PassArgs a{};
        a.seg = p.d_seg;
        a.chunk = p.d_chunk;
        a.piece = p.d_piece;
        a.arena = op->d_arena;
        a.ws = op->d_ws;
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
    if (op->prof_enabled) op->prof_calls.push_back(std::move(ev));
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
// CUDA or library routine.
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
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int rt = rt_for(r);
    const size_t smem = pass_smem_bytes(op, rt);
    {
        const int64_t work = std::max<int64_t>(N * r, (int64_t)op->zero_rows.size() * op->kp * r);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096));
        k_prologue<<<grid, 256, 0, s>>>(u1, ws, op->d_perm, N, r, op->d_zero_rows,
                                        (int)op->zero_rows.size(), op->kp);
        H2_CUDA_TRY(cudaGetLastError());
    }
    for (const Pass& p : op->passes) {
        PassArgs pa{};
        pa.seg = p.d_seg;
        pa.chunk = p.d_chunk;
        pa.piece = p.d_piece;
        pa.arena = op->d_arena;
        pa.ws = ws;
        pa.u2 = u2;
        pa.perm = op->d_perm;
        pa.err = op->d_err;
        pa.N = N;
        pa.nseg = (int)p.seg.size();
        pa.r = r;
        pa.stages = op->stages;
        pa.stage_bytes = op->stage_bytes;
        H2_CUDA_TRY(launch_pass(pa, rt, p.grid, smem, s));
    }
    return H2_OK;
}
