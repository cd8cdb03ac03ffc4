// The finite-element half of the Fredkin-Koehler field evaluation
// (arXiv:1811.05731, Section "Basic Equations"): on a tetrahedral mesh of the
// magnetic body with linear (P1) elements,
//
//  * u1 solves the Poisson problem with Neumann data (Eqs. u1Poiss,
//    u1Neumann); weak form: sum over tetrahedra of int grad u1 . grad v =
//    int M . grad v for every P1 function v, unique up to a constant, fixed
//    here by a zero mean (lumped volume weights, sum_i c_i u1_i = 0);
//  * u2 is harmonic (Eq. u2diri): its boundary values are the boundary
//    integral operator applied to u1 on the boundary (Eq. mainInt; the H2
//    product h2_matvec), its interior values solve the P1 Dirichlet problem;
//  * the energy density in units of K_d = mu0 Ms^2 / 2 is
//    e_d / K_d = (1/V) int M . grad(u1 + u2) dV (Section "Magnetostatic field
//    and energy").
//
// Both linear systems are solved by conjugate gradients with the diagonal
// of the stiffness matrix as preconditioner, in FP64, every step a kernel of
// this file: CSR products (one thread per row), dot products (warp shuffles,
// one atomic addition per CTA) and vector updates.  The scalars of iteration
// i live in slots of their own on the device (no host round trip per
// iteration); the host reads the residual every few iterations to stop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "h2_internal.h"

namespace h2 {
namespace {

constexpr int kFemThreads = 256;
constexpr int kCgCheck = 8;   // iterations between the host's residual checks

__device__ __forceinline__ double warp_sum_f(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
    return v;
}

// Adds the CTA's sum of v into *dst (one atomic addition per CTA).
__device__ __forceinline__ void block_add(double v, double* dst) {
    __shared__ double red[kFemThreads / 32];
    v = warp_sum_f(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kFemThreads / 32; ++i) s += red[i];
        atomicAdd(dst, s);
    }
}

// Volume and the gradients of the four barycentric functions of every
// tetrahedron: with edges e_i = p_i - p_0 and det = e_1 . (e_2 x e_3),
// grad l_1 = e_2 x e_3 / det, grad l_2 = e_3 x e_1 / det, grad l_3 =
// e_1 x e_2 / det, grad l_0 = -(their sum); volume det / 6.
__global__ void k_fem_geom(int64_t nt, const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                           double* __restrict__ vol, double* __restrict__ grad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double p[4][3];
    for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) p[a][d] = xyz[3 * (int64_t)tets[4 * t + a] + d];
    double e[3][3];
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d) e[i][d] = p[i + 1][d] - p[0][d];
    auto cross = [](const double* u, const double* v, double* w) {
        w[0] = u[1] * v[2] - u[2] * v[1];
        w[1] = u[2] * v[0] - u[0] * v[2];
        w[2] = u[0] * v[1] - u[1] * v[0];
    };
    double g[4][3];
    cross(e[1], e[2], g[1]);
    cross(e[2], e[0], g[2]);
    cross(e[0], e[1], g[3]);
    const double det = e[0][0] * g[1][0] + e[0][1] * g[1][1] + e[0][2] * g[1][2];
    for (int i = 1; i < 4; ++i)
        for (int d = 0; d < 3; ++d) g[i][d] /= det;
    for (int d = 0; d < 3; ++d) g[0][d] = -(g[1][d] + g[2][d] + g[3][d]);
    vol[t] = det / 6.0;
    for (int a = 0; a < 4; ++a)
        for (int d = 0; d < 3; ++d) grad[12 * t + 3 * a + d] = g[a][d];
}

// Stiffness entries vol grad l_a . grad l_b added into the CSR values at the
// positions `map` recorded for (tetrahedron, a, b); one thread per entry.
__global__ void k_fem_stiff(int64_t nt, const double* __restrict__ vol, const double* __restrict__ grad,
                            const int32_t* __restrict__ map, double* __restrict__ val) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 16 * nt) return;
    const int64_t t = idx / 16;
    const int a = (int)(idx % 16) / 4, b = (int)(idx % 4);
    const double* g = grad + 12 * t;
    const double v = vol[t] * (g[3 * a] * g[3 * b] + g[3 * a + 1] * g[3 * b + 1] + g[3 * a + 2] * g[3 * b + 2]);
    atomicAdd(val + map[idx], v);
}

// Diagonal of the CSR matrix and the lumped volume weight of every node.
__global__ void k_fem_diag(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const double* __restrict__ val, double* __restrict__ diag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = 0.0;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q)
        if (col[q] == i) d = val[q];
    diag[i] = d;
}

__global__ void k_fem_mass(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ vol,
                           double* __restrict__ mass, double* __restrict__ total) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (t < nt) {
        v = vol[t];
        for (int a = 0; a < 4; ++a) atomicAdd(mass + tets[4 * t + a], 0.25 * v);
    }
    block_add(v, total);
}

// Right-hand side of the Neumann problem: f_i = sum over the tetrahedra at
// node i of vol M_t . grad l_i (M: one vector per tetrahedron).
__global__ void k_fem_rhs_u1(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ vol,
                             const double* __restrict__ grad, const double* __restrict__ M, double* __restrict__ f) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const double* g = grad + 12 * t;
    const double mx = M[3 * t], my = M[3 * t + 1], mz = M[3 * t + 2];
    for (int a = 0; a < 4; ++a)
        atomicAdd(f + tets[4 * t + a], vol[t] * (mx * g[3 * a] + my * g[3 * a + 1] + mz * g[3 * a + 2]));
}

// (1/V) sum over tetrahedra of vol M_t . grad u with u = u1 + u2.
__global__ void k_fem_energy(int64_t nt, const int32_t* __restrict__ tets, const double* __restrict__ vol,
                             const double* __restrict__ grad, const double* __restrict__ M,
                             const double* __restrict__ u1, const double* __restrict__ u2, double* __restrict__ acc) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (t < nt) {
        const double* g = grad + 12 * t;
        double gu[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 4; ++a) {
            const int32_t i = tets[4 * t + a];
            const double u = u1[i] + u2[i];
            for (int d = 0; d < 3; ++d) gu[d] += u * g[3 * a + d];
        }
        e = vol[t] * (M[3 * t] * gu[0] + M[3 * t + 1] * gu[1] + M[3 * t + 2] * gu[2]);
    }
    block_add(e, acc);
}

// ---- conjugate gradients on the rows with mask 1 (mask NULL: every row) ----
// Scalars of iteration it at S[4 it ..]: rz (r . z), pq (p . A p), rr (r . r);
// S[3]: b . b.
__device__ __forceinline__ double row_dot(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                          const double* __restrict__ val, const double* __restrict__ v, int64_t i) {
    double s = 0.0;
    for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) s = fma(val[q], v[col[q]], s);
    return s;
}

// r = mask (b - A x), z = r / diag, p = z; rz_0, rr_0 and b . b.
__global__ void k_cg_init(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const double* __restrict__ val, const unsigned char* __restrict__ mask,
                          const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ r,
                          double* __restrict__ z, double* __restrict__ p, const double* __restrict__ diag,
                          double* __restrict__ S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rz = 0.0, rr = 0.0, bb = 0.0;
    if (i < n) {
        const bool on = !mask || mask[i];
        const double ri = on ? b[i] - row_dot(rowptr, col, val, x, i) : 0.0;
        const double zi = on ? ri / diag[i] : 0.0;
        r[i] = ri;
        z[i] = zi;
        p[i] = zi;
        rz = ri * zi;
        rr = ri * ri;
        bb = on ? b[i] * b[i] : 0.0;
    }
    block_add(rz, S + 0);
    __syncthreads();
    block_add(rr, S + 2);
    __syncthreads();
    block_add(bb, S + 3);
}

// The iteration kernels read the iteration number it from cnt[0] (so that
// a captured sequence of iterations can be replayed): k_cg_dir's last CTA
// advances it.  They loop over their rows with a grid stride, so that a grid
// of a few hundred CTAs makes each reduction a few hundred atomic additions.

// q = mask A p; pq_it = p . q (one thread per row: measured faster than
// several lanes per row, whose rows of about 15 entries leave lanes idle).
__global__ void k_cg_q(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const unsigned char* __restrict__ mask,
                       const double* __restrict__ p, double* __restrict__ q, double* __restrict__ S,
                       const int32_t* __restrict__ cnt) {
    const int it = cnt[0];
    double pq = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double qi = (!mask || mask[i]) ? row_dot(rowptr, col, val, p, i) : 0.0;
        q[i] = qi;
        pq += p[i] * qi;
    }
    block_add(pq, S + 4 * (int64_t)it + 1);
}

// alpha = rz_it / pq_it; x += alpha p; r -= alpha q; z = r / diag; rz, rr of it + 1.
__global__ void k_cg_update(int64_t n, const unsigned char* __restrict__ mask, const double* __restrict__ diag,
                            double* __restrict__ x, double* __restrict__ r, double* __restrict__ z,
                            const double* __restrict__ p, const double* __restrict__ q, double* __restrict__ S,
                            const int32_t* __restrict__ cnt) {
    const int it = cnt[0];
    const double pq = S[4 * (int64_t)it + 1];
    const double alpha = pq != 0.0 ? S[4 * (int64_t)it] / pq : 0.0;
    double rz = 0.0, rr = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        const double zi = (!mask || mask[i]) ? ri / diag[i] : 0.0;
        r[i] = ri;
        z[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
    }
    block_add(rz, S + 4 * (int64_t)(it + 1));
    __syncthreads();
    block_add(rr, S + 4 * (int64_t)(it + 1) + 2);
}

// beta = rz_{it+1} / rz_it; p = z + beta p; the last CTA to finish advances
// the iteration number (every CTA has read it by then).
__global__ void k_cg_dir(int64_t n, double* __restrict__ p, const double* __restrict__ z, const double* __restrict__ S,
                         int32_t* __restrict__ cnt) {
    const int it = cnt[0];
    const double rz0 = S[4 * (int64_t)it];
    const double beta = rz0 != 0.0 ? S[4 * (int64_t)(it + 1)] / rz0 : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(cnt + 1, 1) == (int)gridDim.x - 1) {
            cnt[1] = 0;
            cnt[0] = it + 1;
            __threadfence();
        }
    }
}

// *acc += sum_i w_i x_i (w NULL: all ones)
__global__ void k_fem_wdot(int64_t n, const double* __restrict__ w, const double* __restrict__ x, double* __restrict__ acc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    block_add(i < n ? (w ? w[i] : 1.0) * x[i] : 0.0, acc);
}

// x -= (*num) / n
__global__ void k_fem_center(int64_t n, double* __restrict__ x, const double* __restrict__ num) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] -= *num / (double)n;
}

// x -= (*num) / (*den)
__global__ void k_fem_shift(int64_t n, double* __restrict__ x, const double* __restrict__ num,
                            const double* __restrict__ den) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] -= *num / *den;
}

__global__ void k_fem_gather(int64_t ns, const int32_t* __restrict__ surf, const double* __restrict__ u,
                             double* __restrict__ ub) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) ub[i] = u[surf[i]];
}

__global__ void k_fem_scatter(int64_t ns, const int32_t* __restrict__ surf, const double* __restrict__ ub,
                              double* __restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ns) u[surf[i]] = ub[i];
}

// b = -mask (A uB): the Dirichlet problem's right-hand side on the interior rows.
__global__ void k_fem_dirichlet_rhs(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, const unsigned char* __restrict__ mask,
                                    const double* __restrict__ uB, double* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = mask[i] ? -row_dot(rowptr, col, val, uB, i) : 0.0;
}

}  // namespace

// Device data of a tetrahedral mesh (handle kind 3).
struct FemData {
    int64_t nv = 0, nt = 0, ns = 0, nnz = 0;
    double volume = 0.0;
    double *xyz = nullptr, *vol = nullptr, *grad = nullptr, *val = nullptr, *diag = nullptr, *mass = nullptr;
    double* scal = nullptr;   // the volume, then scratch scalars
    int32_t *tets = nullptr, *surf = nullptr, *rowptr = nullptr, *col = nullptr, *map = nullptr;
    unsigned char* interior = nullptr;
};

void fem_release(FemData* f) {
    if (!f) return;
    for (void* p : {(void*)f->xyz, (void*)f->vol, (void*)f->grad, (void*)f->val, (void*)f->diag, (void*)f->mass,
                    (void*)f->scal, (void*)f->tets, (void*)f->surf, (void*)f->rowptr, (void*)f->col, (void*)f->map,
                    (void*)f->interior})
        if (p) cudaFree(p);
    delete f;
}

namespace {
template <class T>
int fem_upload(const std::vector<T>& v, T** d) {
    H2_CUDA_TRY(cudaMalloc((void**)d, sizeof(T) * std::max<size_t>(1, v.size())));
    if (!v.empty()) H2_CUDA_TRY(cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
    return H2_OK;
}
inline unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kFemThreads - 1) / kFemThreads); }
// CTAs of the iteration kernels (grid-stride loops): two per SM; measured
// faster than a CTA per 256 rows (more same-address atomic additions per
// reduction) on balls of 36k-275k nodes
constexpr unsigned kCgCtas = 304;
inline unsigned cg_grid(int64_t rows) { return std::min<unsigned>(grid_of(rows), kCgCtas); }

// Preconditioned conjugate gradients for A x = b on the rows with mask 1
// (mask NULL: all), x starting from its content; stops when |r| <= tol |b|
// (checked every kCgCheck iterations) or after max_iter iterations.  The
// iterations run as a CUDA graph of kCgCheck of them (captured on a stream of
// its own, replayed on s): the host reads one residual per replay.
int fem_cg(const FemData& F, const unsigned char* mask, const double* b, double* x, double* work, double tol,
           int max_iter, cudaStream_t s, int* iters, double* resid) {
    const int64_t n = F.nv;
    double *r = work, *z = work + n, *p = work + 2 * n, *q = work + 3 * n;
    double* S = nullptr;
    int32_t* cnt = nullptr;
    const size_t nscal = 4 * ((size_t)max_iter + 2);
    H2_CUDA_TRY(cudaMalloc((void**)&S, sizeof(double) * nscal));
    cudaError_t e = cudaMalloc((void**)&cnt, sizeof(int32_t) * 2);
    if (e == cudaSuccess) e = cudaMemsetAsync(S, 0, sizeof(double) * nscal, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 2, s);
    const unsigned gv = cg_grid(n);
    auto iteration = [&](cudaStream_t t) {
        k_cg_q<<<gv, kFemThreads, 0, t>>>(n, F.rowptr, F.col, F.val, mask, p, q, S, cnt);
        k_cg_update<<<gv, kFemThreads, 0, t>>>(n, mask, F.diag, x, r, z, p, q, S, cnt);
        k_cg_dir<<<gv, kFemThreads, 0, t>>>(n, p, z, S, cnt);
    };
    if (e == cudaSuccess) {
        k_cg_init<<<grid_of(n), kFemThreads, 0, s>>>(n, F.rowptr, F.col, F.val, mask, b, x, r, z, p, F.diag, S);
        e = cudaGetLastError();
    }
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && max_iter >= kCgCheck) {
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < kCgCheck; ++k) iteration(cs);
            const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            e = e2 != cudaSuccess ? e2 : cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    }
    double h0[4] = {0.0, 0.0, 0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h0, S, sizeof(h0), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const double bnorm = sqrt(h0[3]);
    int it = 0;
    double rel = bnorm > 0.0 ? sqrt(h0[2]) / bnorm : 0.0;
    while (e == cudaSuccess && rel > tol && it < max_iter) {
        if (max_iter - it >= kCgCheck) {
            e = cudaGraphLaunch(exec, s);
            it += kCgCheck;
        } else {   // the last iterations below a whole replay
            for (; it < max_iter; ++it) iteration(s);
            e = cudaGetLastError();
        }
        double rr = 0.0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&rr, S + 4 * (size_t)it + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        rel = sqrt(rr) / bnorm;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cs) cudaStreamDestroy(cs);
    cudaStreamSynchronize(s);
    cudaFree(S);
    cudaFree(cnt);
    if (e != cudaSuccess) {
        set_cuda_error(e, "conjugate gradients", __FILE__, __LINE__);
        return H2_ERR_CUDA;
    }
    *iters = it;
    *resid = rel;
    return H2_OK;
}
}  // namespace
}  // namespace h2

using h2::FemData;

extern "C" int h2_fem_create(const double* xyz, int64_t n_vertices, const int32_t* tets, int64_t n_tets,
                             const int32_t* surf_nodes, int64_t n_surf, h2_handle** out_fem) {
    using namespace h2;
    if (!xyz || !tets || !surf_nodes || !out_fem || n_vertices < 4 || n_tets < 1 || n_surf < 4 ||
        n_surf > n_vertices || n_vertices > INT32_MAX || 16 * n_tets > INT32_MAX)
        return H2_ERR_INVALID_ARG;
    *out_fem = nullptr;
    std::vector<char> is_surf((size_t)n_vertices, 0);
    for (int64_t i = 0; i < n_surf; ++i) {
        const int32_t v = surf_nodes[i];
        if (v < 0 || v >= n_vertices || is_surf[v]) return H2_ERR_INVALID_ARG;
        is_surf[v] = 1;
    }
    // orientation: every tetrahedron of positive volume (the gradients assume it)
    for (int64_t t = 0; t < n_tets; ++t) {
        const int32_t* q = tets + 4 * t;
        for (int a = 0; a < 4; ++a)
            if (q[a] < 0 || q[a] >= n_vertices) return H2_ERR_INVALID_ARG;
        double e[3][3];
        for (int i = 0; i < 3; ++i)
            for (int d = 0; d < 3; ++d) e[i][d] = xyz[3 * (int64_t)q[i + 1] + d] - xyz[3 * (int64_t)q[0] + d];
        const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                           e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
        if (!(det > 0.0)) return H2_ERR_MESH_ORIENTATION;
    }
    // CSR pattern of the P1 stiffness matrix and every tetrahedron's 16 positions in it
    std::vector<std::vector<int32_t>> nb((size_t)n_vertices);
    for (int64_t t = 0; t < n_tets; ++t)
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) nb[tets[4 * t + a]].push_back(tets[4 * t + b]);
    std::vector<int32_t> rowptr((size_t)n_vertices + 1, 0), col;
    for (int64_t i = 0; i < n_vertices; ++i) {
        std::sort(nb[i].begin(), nb[i].end());
        nb[i].erase(std::unique(nb[i].begin(), nb[i].end()), nb[i].end());
        rowptr[i + 1] = rowptr[i] + (int32_t)nb[i].size();
        col.insert(col.end(), nb[i].begin(), nb[i].end());
    }
    std::vector<int32_t> map((size_t)16 * n_tets);
    for (int64_t t = 0; t < n_tets; ++t)
        for (int a = 0; a < 4; ++a) {
            const int32_t i = tets[4 * t + a];
            for (int b = 0; b < 4; ++b) {
                const auto it = std::lower_bound(col.begin() + rowptr[i], col.begin() + rowptr[i + 1], tets[4 * t + b]);
                map[16 * t + 4 * a + b] = (int32_t)(it - col.begin());
            }
        }
    std::vector<unsigned char> interior((size_t)n_vertices);
    for (int64_t i = 0; i < n_vertices; ++i) interior[i] = is_surf[i] ? 0 : 1;
    auto* F = new FemData();
    F->nv = n_vertices;
    F->nt = n_tets;
    F->ns = n_surf;
    F->nnz = (int64_t)col.size();
    int rc = H2_OK;
    auto fail = [&](int code) {
        fem_release(F);
        return code;
    };
    if ((rc = fem_upload(std::vector<double>(xyz, xyz + 3 * n_vertices), &F->xyz)) ||
        (rc = fem_upload(std::vector<int32_t>(tets, tets + 4 * n_tets), &F->tets)) ||
        (rc = fem_upload(std::vector<int32_t>(surf_nodes, surf_nodes + n_surf), &F->surf)) ||
        (rc = fem_upload(rowptr, &F->rowptr)) || (rc = fem_upload(col, &F->col)) || (rc = fem_upload(map, &F->map)) ||
        (rc = fem_upload(interior, &F->interior)))
        return fail(rc);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](double** p, size_t n) {
        if (e == cudaSuccess) e = cudaMalloc((void**)p, sizeof(double) * std::max<size_t>(1, n));
        if (e == cudaSuccess) e = cudaMemset(*p, 0, sizeof(double) * std::max<size_t>(1, n));
    };
    alloc(&F->vol, n_tets);
    alloc(&F->grad, 12 * (size_t)n_tets);
    alloc(&F->val, col.size());
    alloc(&F->diag, n_vertices);
    alloc(&F->mass, n_vertices);
    alloc(&F->scal, 16);
    if (e != cudaSuccess) {
        set_cuda_error(e, "h2_fem_create", __FILE__, __LINE__);
        return fail(e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA);
    }
    k_fem_geom<<<grid_of(n_tets), kFemThreads>>>(n_tets, F->xyz, F->tets, F->vol, F->grad);
    k_fem_stiff<<<grid_of(16 * n_tets), kFemThreads>>>(n_tets, F->vol, F->grad, F->map, F->val);
    k_fem_diag<<<grid_of(n_vertices), kFemThreads>>>(n_vertices, F->rowptr, F->col, F->val, F->diag);
    k_fem_mass<<<grid_of(n_tets), kFemThreads>>>(n_tets, F->tets, F->vol, F->mass, F->scal);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&F->volume, F->scal, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        set_cuda_error(e, "h2_fem_create kernels", __FILE__, __LINE__);
        return fail(H2_ERR_CUDA);
    }
    auto* h = new h2_handle();
    h->kind = 3;
    h->fem = F;
    cudaGetDevice(&h->device);
    *out_fem = h;
    return H2_OK;
}

extern "C" int h2_fem_solve(h2_handle* fem, h2_handle* op, const double* M, double* u1, double* u2, double tol,
                            int32_t max_iter, void* cuda_stream, h2_fem_report_t* out) {
    using namespace h2;
    if (!fem || !op || !M || !u1 || !u2 || !(tol > 0.0) || max_iter < 1) return H2_ERR_INVALID_ARG;
    if (fem->kind != 3 || op->kind != 2) return H2_ERR_WRONG_HANDLE;
    const FemData& F = *fem->fem;
    if (op->geom->N != F.ns || op->device != fem->device) return H2_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t n = F.nv, ns = F.ns;
    // scratch: f, uB (boundary values), b, four CG vectors, u1 and u2 on the boundary, scalars
    double* w = nullptr;
    const size_t nw = 7 * (size_t)n + 2 * (size_t)ns + 8;
    H2_CUDA_TRY(cudaMalloc((void**)&w, sizeof(double) * nw));
    double *f = w, *uB = w + n, *b = w + 2 * n, *cg = w + 3 * n, *u1b = w + 7 * n, *u2b = u1b + ns, *sc = u2b + ns;
    int rc = H2_OK;
    h2_fem_report_t rep{};
    cudaError_t e = cudaMemsetAsync(w, 0, sizeof(double) * nw, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(u1, 0, sizeof(double) * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(u2, 0, sizeof(double) * n, s);
    if (e != cudaSuccess) rc = H2_ERR_CUDA;
    // u1: Neumann problem, then the constant that gives it zero (lumped) mean
    if (rc == H2_OK) {
        k_fem_rhs_u1<<<grid_of(F.nt), kFemThreads, 0, s>>>(F.nt, F.tets, F.vol, F.grad, M, f);
        // the stiffness matrix annihilates constants: f's sum (zero up to
        // rounding) is removed, so that f lies in its range
        k_fem_wdot<<<grid_of(n), kFemThreads, 0, s>>>(n, nullptr, f, sc + 2);
        k_fem_center<<<grid_of(n), kFemThreads, 0, s>>>(n, f, sc + 2);
        rc = fem_cg(F, nullptr, f, u1, cg, tol, max_iter, s, &rep.iters_u1, &rep.resid_u1);
    }
    if (rc == H2_OK) {
        k_fem_wdot<<<grid_of(n), kFemThreads, 0, s>>>(n, F.mass, u1, sc);
        k_fem_shift<<<grid_of(n), kFemThreads, 0, s>>>(n, u1, sc, F.scal);
        // u2 on the boundary: the H2 product of the double-layer operator with u1|boundary
        k_fem_gather<<<grid_of(ns), kFemThreads, 0, s>>>(ns, F.surf, u1, u1b);
        if ((e = cudaGetLastError()) != cudaSuccess) rc = H2_ERR_CUDA;
    }
    if (rc == H2_OK) rc = matvec_device(op, u1b, u2b, 1, s);
    if (rc == H2_OK) {
        // u2 inside: the Dirichlet problem A_II x_I = -A_IB u2_B, u2 = u2_B + x
        k_fem_scatter<<<grid_of(ns), kFemThreads, 0, s>>>(ns, F.surf, u2b, uB);
        k_fem_dirichlet_rhs<<<grid_of(n), kFemThreads, 0, s>>>(n, F.rowptr, F.col, F.val, F.interior, uB, b);
        rc = fem_cg(F, F.interior, b, u2, cg, tol, max_iter, s, &rep.iters_u2, &rep.resid_u2);
    }
    if (rc == H2_OK) {
        k_fem_scatter<<<grid_of(ns), kFemThreads, 0, s>>>(ns, F.surf, u2b, u2);
        k_fem_energy<<<grid_of(F.nt), kFemThreads, 0, s>>>(F.nt, F.tets, F.vol, F.grad, M, u1, u2, sc + 1);
        double acc = 0.0;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = H2_ERR_CUDA;
        rep.volume = F.volume;
        rep.energy = acc / F.volume;
    }
    if (rc == H2_ERR_CUDA && e != cudaSuccess) set_cuda_error(e, "h2_fem_solve", __FILE__, __LINE__);
    cudaStreamSynchronize(s);
    cudaFree(w);
    if (rc == H2_OK && out) *out = rep;
    return rc;
}
