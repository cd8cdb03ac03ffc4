// Algebraic recompression of the interpolation H2 operator on the device
// (arXiv:1811.05731, Section "H2-Matrix Compression": the cluster bases of
// the approximation are compressed algebraically, after the construction,
// with a relative truncation threshold).  The steps are the published ones
// for nested bases (S. Boerm, Efficient Numerical Methods for Non-local
// Operators, EMS 2010: orthogonalisation of nested cluster bases, and their
// compression with total cluster-basis weights), each done for the row
// bases (V, transfers E, the target side of the blocks) and for the column
// bases (W, the source side):
//
//  1. Orthogonalisation, leaves to root: V_t = Q_t R_t (thin QR) at the
//     leaves; a parent factorises its children's R_c E_c stacked,
//     [R_c0 E_c0; R_c1 E_c1] = Qhat R_t, Qhat's rows being the nested
//     transfers of the orthonormal basis.  Couplings become
//     S'_ts = R_t S_ts R_s^T (row R of t, column R of s).
//  2. Total weights, root to leaves: the far-field rows of t in Q_t
//     coordinates span [S'_ts for the blocks of t, Qhat_t Z_parent]; Z_t is a
//     matrix of at most q_t columns with the same Gram matrix, condensed one
//     block at a time by QR of the transpose (Z = R^T).
//  3. Truncation, leaves to root: G_t = I at a leaf, [B_c0 Qhat_c0;
//     B_c1 Qhat_c1] at a parent; the left singular vectors X_t of G_t Z_t
//     whose singular values exceed eps times the largest; new leaf basis
//     Q_t X_t, new transfers the children's rows of X_t, B_t = X_t^T G_t.
//  4. New couplings B_t S'_ts B'_s^T.
//
// Everything is FP64.  One CTA (256 threads) per cluster or block does its
// small dense factorisations in global memory (they stay in L1/L2): Householder
// QR (Golub-Van Loan, Algorithm 5.2.1), explicit thin Q by backward
// accumulation, one-sided Jacobi SVD (Hestenes; Demmel-Veselic ordering
// by a round-robin tournament), plain matrix products.  All matrices are
// column-major.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "h2_internal.h"

namespace h2 {
namespace {

constexpr int kLaThreads = 256;
constexpr int kLaWarps = kLaThreads / 32;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
    return v;
}

// Sum over the CTA (every thread gets the result); `red` holds kLaWarps doubles.
__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < kLaWarps; ++i) s += red[i];
    return s;
}

// Householder QR in place of the m x n matrix A (leading dimension lda):
// on return its upper triangle holds R (p = min(m, n) rows), column j below
// the diagonal the Householder vector v_j with v_j[0] = 1 implicit, and
// beta[j] the reflector's factor (H_j = I - beta_j v_j v_j^T; beta_j = 0:
// no reflection).  Golub-Van Loan's stable choice of v_j[0].
__device__ void cta_qr(double* A, int lda, int m, int n, double* beta, double* red) {
    const int p = m < n ? m : n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = 0; j < p; ++j) {
        double* aj = A + (size_t)j * lda;
        double part = 0.0;
        for (int i = j + 1 + threadIdx.x; i < m; i += kLaThreads) part += aj[i] * aj[i];
        const double sigma = block_sum(part, red);
        const double x0 = aj[j];
        double b = 0.0, v0 = 1.0, mu = x0;
        if (sigma > 0.0 || x0 < 0.0) {
            mu = sqrt(x0 * x0 + sigma);
            v0 = x0 <= 0.0 ? x0 - mu : -sigma / (x0 + mu);
            b = 2.0 * v0 * v0 / (sigma + v0 * v0);
        }
        __syncthreads();
        if (b != 0.0)
            for (int i = j + 1 + threadIdx.x; i < m; i += kLaThreads) aj[i] /= v0;
        if (threadIdx.x == 0) {
            aj[j] = mu;
            beta[j] = b;
        }
        __syncthreads();
        if (b != 0.0) {
            // trailing columns: c -= b v (v . c), one warp per column
            for (int c = j + 1 + warp; c < n; c += kLaWarps) {
                double* ac = A + (size_t)c * lda;
                double d = lane == 0 ? ac[j] : 0.0;
                for (int i = j + 1 + lane; i < m; i += 32) d += aj[i] * ac[i];
                d = warp_sum(d) * b;
                if (lane == 0) ac[j] -= d;
                for (int i = j + 1 + lane; i < m; i += 32) ac[i] -= d * aj[i];
            }
        }
        __syncthreads();
    }
}

// The first q columns of Q = H_0 H_1 ... H_{p-1} (m x q, leading dimension
// ldq) from the reflectors cta_qr left in A, by backward accumulation.
__device__ void cta_form_q(const double* A, int lda, int m, int n, const double* beta, double* Q, int ldq, int q) {
    const int p = m < n ? m : n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int c = 0; c < q; ++c)
        for (int i = threadIdx.x; i < m; i += kLaThreads) Q[(size_t)c * ldq + i] = i == c ? 1.0 : 0.0;
    __syncthreads();
    for (int j = p - 1; j >= 0; --j) {
        const double b = beta[j];
        if (b == 0.0) continue;
        const double* aj = A + (size_t)j * lda;
        for (int c = j + warp; c < q; c += kLaWarps) {   // columns below j are e_c, untouched
            double* qc = Q + (size_t)c * ldq;
            double d = lane == 0 ? qc[j] : 0.0;
            for (int i = j + 1 + lane; i < m; i += 32) d += aj[i] * qc[i];
            d = warp_sum(d) * b;
            if (lane == 0) qc[j] -= d;
            for (int i = j + 1 + lane; i < m; i += 32) qc[i] -= d * aj[i];
        }
        __syncthreads();
    }
}

// C (m x n, ldc) = op(A) op(B) with op(X) = X or X^T; A is m x k after op,
// B is k x n after op.  Threads over the entries of C.
__device__ void cta_gemm(double* C, int ldc, const double* A, int lda, bool ta, const double* B, int ldb, bool tb,
                         int m, int n, int k) {
    for (int idx = threadIdx.x; idx < m * n; idx += kLaThreads) {
        const int i = idx % m, j = idx / m;
        double s = 0.0;
        for (int l = 0; l < k; ++l) {
            const double a = ta ? A[(size_t)i * lda + l] : A[(size_t)l * lda + i];
            const double bb = tb ? B[(size_t)l * ldb + j] : B[(size_t)j * ldb + l];
            s = fma(a, bb, s);
        }
        C[(size_t)j * ldc + i] = s;
    }
}

// One-sided Jacobi (Hestenes) on the columns of the a x z matrix U (ldu):
// rotations of column pairs, in round-robin tournament order, until every
// pair is orthogonal to 1e-15 of the product of its norms (at most 60
// sweeps).  On return U's columns are orthogonal, sv[j] = |U_j|, and
// order[0..z) lists the columns by decreasing sv.  `flag` is one int of
// shared memory.
__device__ void cta_jacobi(double* U, int ldu, int a, int z, double* sv, int* order, int* flag) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ze = z + (z & 1);   // even, with a dummy column past z
    for (int sweep = 0; sweep < 60 && z > 1; ++sweep) {
        if (threadIdx.x == 0) *flag = 0;
        __syncthreads();
        for (int round = 0; round < ze - 1; ++round) {
            for (int k = warp; k < ze / 2; k += kLaWarps) {
                // circle method: position 0 fixed, the others rotate
                auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (ze - 1); };
                int p = at(k), q = at(ze - 1 - k);
                if (p >= z || q >= z) continue;
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                double* up = U + (size_t)p * ldu;
                double* uq = U + (size_t)q * ldu;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < a; i += 32) {
                    al += up[i] * up[i];
                    be += uq[i] * uq[i];
                    ga += up[i] * uq[i];
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int i = lane; i < a; i += 32) {
                    const double x = up[i], y = uq[i];
                    up[i] = c * x - s * y;
                    uq[i] = s * x + c * y;
                }
                if (lane == 0) *flag = 1;
            }
            __syncthreads();
        }
        const int rotated = *flag;
        __syncthreads();
        if (!rotated) break;
    }
    for (int j = warp; j < z; j += kLaWarps) {
        double s = 0.0;
        for (int i = lane; i < a; i += 32) s += U[(size_t)j * ldu + i] * U[(size_t)j * ldu + i];
        s = warp_sum(s);
        if (lane == 0) sv[j] = sqrt(s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // z <= 2 H2_MAX_K: insertion sort by decreasing value
        for (int j = 0; j < z; ++j) order[j] = j;
        for (int j = 1; j < z; ++j) {
            const int v = order[j];
            int i = j - 1;
            while (i >= 0 && sv[order[i]] < sv[v]) {
                order[i + 1] = order[i];
                --i;
            }
            order[i + 1] = v;
        }
    }
    __syncthreads();
}

// One side (row bases or column bases) of one cluster.  Offsets `R`..`work`
// count doubles in the recompression pool; `in` and `E` are byte offsets in
// the FP64 interpolation arena.
struct RcNode {
    int32_t leaf, size, q, qa, qb;   // q: rank after orthogonalisation; qa, qb: the children's
    int32_t child0, child1, parent, second;   // second: this cluster is its parent's child1
    int32_t blk0, nblk;              // this side's far blocks (indices into the block list)
    int64_t in;                      // leaf: its interpolation basis; -1 otherwise
    int64_t E;                       // its transfer E_c (k x k, child x parent); -1 at the root
    int64_t R, Q, Z, B, N, work;
};

// 1. Orthogonalisation of one level (bottom up): a leaf factorises its basis
// (rows: V_t, |t| x k column-major; columns: W_t, stored k x |t| column-major,
// read transposed); a parent the stacked [R_c0 E_c0; R_c1 E_c1].  Writes R
// (q x k, ld q) and the thin Q (leaf: |t| x q, ld |t|; parent: the stacked
// (qa + qb) x q, ld qa + qb, whose row blocks are the children's transfers).
__global__ void __launch_bounds__(kLaThreads) k_rc_orth(const RcNode* __restrict__ nodes, const int32_t* __restrict__ list,
                                                        int side, const unsigned char* __restrict__ arena,
                                                        double* __restrict__ pool, int k) {
    __shared__ double beta[2 * H2_MAX_K];
    __shared__ double red[kLaWarps];
    const RcNode n = nodes[list[blockIdx.x]];
    double* W = pool + n.work;
    int m;
    if (n.leaf) {
        m = n.size;
        const double* src = reinterpret_cast<const double*>(arena + n.in);
        for (int idx = threadIdx.x; idx < m * k; idx += kLaThreads) {
            const int i = idx % m, mu = idx / m;
            W[idx] = side == 0 ? src[idx] : src[(size_t)i * k + mu];
        }
    } else {
        const RcNode a = nodes[n.child0], b = nodes[n.child1];
        m = a.q + b.q;
        cta_gemm(W, m, pool + a.R, a.q, false, reinterpret_cast<const double*>(arena + a.E), k, false, a.q, k, k);
        cta_gemm(W + a.q, m, pool + b.R, b.q, false, reinterpret_cast<const double*>(arena + b.E), k, false, b.q, k,
                 k);
    }
    __syncthreads();
    cta_qr(W, m, m, k, beta, red);
    const int q = n.q;
    double* R = pool + n.R;
    for (int idx = threadIdx.x; idx < q * k; idx += kLaThreads) {
        const int i = idx % q, j = idx / q;
        R[idx] = i <= j ? W[(size_t)j * m + i] : 0.0;
    }
    __syncthreads();
    cta_form_q(W, m, m, k, beta, pool + n.Q, m, q);
}

// S'_ts = R_t S_ts R_s^T (row R of the target, column R of the source),
// written over S_ts (q_t x q_s, ld q_t).  `temp`: k x k doubles per CTA.
__global__ void __launch_bounds__(kLaThreads) k_rc_sprime(const int2* __restrict__ blk, const int64_t* __restrict__ soff,
                                                          int b0, int nb, const RcNode* __restrict__ rows,
                                                          const RcNode* __restrict__ cols, unsigned char* arena,
                                                          const double* __restrict__ pool, double* __restrict__ temp,
                                                          int k) {
    const int b = b0 + blockIdx.x;
    if (b >= nb) return;
    const int t = blk[b].x, s = blk[b].y;
    double* S = reinterpret_cast<double*>(arena + soff[b]);
    double* T = temp + (size_t)blockIdx.x * k * k;
    const int qt = rows[t].q, qs = cols[s].q;
    cta_gemm(T, k, S, k, false, pool + cols[s].R, qs, true, k, qs, k);
    __syncthreads();
    cta_gemm(S, qt, pool + rows[t].R, qt, false, T, k, false, qt, qs, k);
}

// Z (q x q, ld q) = R^T from the QR of the m x q matrix T (ld m, m >= q).
__device__ void condense_into(double* Z, int q, double* T, int m, double* beta, double* red) {
    cta_qr(T, m, m, q, beta, red);
    for (int idx = threadIdx.x; idx < q * q; idx += kLaThreads) {
        const int i = idx % q, j = idx / q;
        Z[idx] = j <= i ? T[(size_t)i * m + j] : 0.0;
    }
    __syncthreads();
}

// 2. Total weights of one level (top down).  The far field reaching cluster c
// in its Q coordinates is [its blocks' S' (rows) or S'^T (columns), Qhat_c
// Z_parent]; Z_c keeps at most q columns with the same Gram matrix: columns
// are appended while they fit and condensed by QR of the transpose when not.
__global__ void __launch_bounds__(kLaThreads) k_rc_weights(const RcNode* __restrict__ nodes, const RcNode* __restrict__ other,
                                                           const int32_t* __restrict__ list, int side,
                                                           const int32_t* __restrict__ blist, const int2* __restrict__ blk,
                                                           const int64_t* __restrict__ soff,
                                                           const unsigned char* __restrict__ arena,
                                                           double* __restrict__ pool, int32_t* __restrict__ zc) {
    __shared__ double beta[2 * H2_MAX_K];
    __shared__ double red[kLaWarps];
    const int c = list[blockIdx.x];
    const RcNode n = nodes[c];
    const int q = n.q;
    double* Z = pool + n.Z;
    double* T = pool + n.work;
    int z = 0;
    if (n.parent >= 0 && zc[n.parent] > 0) {
        const RcNode p = nodes[n.parent];
        const int zp = zc[n.parent], ldq = p.qa + p.qb;
        const double* Qh = pool + p.Q + (n.second ? p.qa : 0);   // this child's rows of the parent's Qhat
        if (zp <= q) {
            cta_gemm(Z, q, Qh, ldq, false, pool + p.Z, p.q, false, q, zp, p.q);
            z = zp;
            __syncthreads();
        } else {   // (Qhat Z_p)^T = Z_p^T Qhat^T, zp x q, then condensed
            cta_gemm(T, zp, pool + p.Z, p.q, true, Qh, ldq, true, zp, q, p.q);
            __syncthreads();
            condense_into(Z, q, T, zp, beta, red);
            z = q;
        }
    }
    for (int e = n.blk0; e < n.blk0 + n.nblk; ++e) {
        const int b = blist[e];
        const double* Sp = reinterpret_cast<const double*>(arena + soff[b]);
        // C = S'_b (q x q_s, ld q) for rows; S'_b^T (S' is q_t x q, ld q_t) for columns
        const int ncol = side == 0 ? other[blk[b].y].q : other[blk[b].x].q;
        const int ldsp = side == 0 ? q : ncol;
        if (z + ncol <= q) {
            for (int idx = threadIdx.x; idx < q * ncol; idx += kLaThreads) {
                const int i = idx % q, j = idx / q;
                Z[(size_t)(z + j) * q + i] = side == 0 ? Sp[(size_t)j * ldsp + i] : Sp[(size_t)i * ldsp + j];
            }
            z += ncol;
            __syncthreads();
        } else {   // T = [Z | C]^T ((z + ncol) x q), condensed into Z
            const int m = z + ncol;
            for (int idx = threadIdx.x; idx < m * q; idx += kLaThreads) {
                const int i = idx % m, j = idx / m;   // T(i, j) = [Z | C](j, i)
                double v;
                if (i < z) v = Z[(size_t)i * q + j];
                else v = side == 0 ? Sp[(size_t)(i - z) * ldsp + j] : Sp[(size_t)j * ldsp + (i - z)];
                T[idx] = v;
            }
            __syncthreads();
            condense_into(Z, q, T, m, beta, red);
            z = q;
        }
    }
    if (threadIdx.x == 0) zc[c] = z;
}

// 3. Truncation of one level (bottom up).  G = I at a leaf, [B_c0 Qhat_c0;
// B_c1 Qhat_c1] at a parent (a = rank_c0 + rank_c1 rows); the left singular
// vectors of G Z whose singular values exceed eps times the largest are X;
// rank = their count (at least one where the cluster's weight is not zero);
// B = X^T G (rank x q, ld q).  A leaf's new basis Q X goes to N (|t| x rank,
// ld |t|), a parent's X to N (a x rank, ld a): rows [0, rank_c0) are the
// first child's new transfer, the rest the second's.
__global__ void __launch_bounds__(kLaThreads) k_rc_truncate(const RcNode* __restrict__ nodes,
                                                            const int32_t* __restrict__ list, double* __restrict__ pool,
                                                            const int32_t* __restrict__ zc, int32_t* __restrict__ rank,
                                                            double eps) {
    __shared__ double sv[H2_MAX_K];
    __shared__ int order[H2_MAX_K];
    __shared__ int flag;
    const int c = list[blockIdx.x];
    const RcNode n = nodes[c];
    const int q = n.q, z = zc[c];
    double* G = pool + n.work;
    int a = q;
    if (!n.leaf) {
        const RcNode A = nodes[n.child0], Bn = nodes[n.child1];
        const int ka = rank[n.child0], kb = rank[n.child1];
        a = ka + kb;
        const int ldq = n.qa + n.qb;
        cta_gemm(G, a, pool + A.B, A.q, false, pool + n.Q, ldq, false, ka, q, A.q);
        cta_gemm(G + ka, a, pool + Bn.B, Bn.q, false, pool + n.Q + n.qa, ldq, false, kb, q, Bn.q);
        __syncthreads();
    }
    double* U = G + (size_t)a * q;   // a x z, ld a
    if (n.leaf) {
        for (int idx = threadIdx.x; idx < q * z; idx += kLaThreads) U[idx] = pool[n.Z + idx];
    } else {
        cta_gemm(U, a, G, a, false, pool + n.Z, q, false, a, z, q);
    }
    __syncthreads();
    int keep = 0;
    if (z > 0 && a > 0) {
        cta_jacobi(U, a, a, z, sv, order, &flag);
        const double smax = sv[order[0]];
        if (smax > 0.0) {
            keep = 1;
            while (keep < z && keep < a && sv[order[keep]] > eps * smax) ++keep;
        }
    }
    // X (a x keep): the kept columns of U, normalised, in decreasing order
    double* X = n.leaf ? U + (size_t)a * z : pool + n.N;
    for (int idx = threadIdx.x; idx < a * keep; idx += kLaThreads) {
        const int i = idx % a, j = idx / a;
        X[idx] = U[(size_t)order[j] * a + i] / sv[order[j]];
    }
    __syncthreads();
    double* B = pool + n.B;
    if (n.leaf) {
        for (int idx = threadIdx.x; idx < keep * q; idx += kLaThreads) {   // B = X^T
            const int i = idx % keep, j = idx / keep;
            B[(size_t)j * q + i] = X[(size_t)i * a + j];
        }
        cta_gemm(pool + n.N, n.size, pool + n.Q, n.size, false, X, a, false, n.size, keep, q);   // Q X
    } else {
        cta_gemm(B, q, X, a, true, G, a, false, keep, q, a);
    }
    if (threadIdx.x == 0) rank[c] = keep;
}

// 4. New couplings S'' = B_t S' B_s^T (rank_t x rank_s, ld rank_t), written
// over S'.  `temp`: k x k doubles per CTA.
__global__ void __launch_bounds__(kLaThreads) k_rc_snew(const int2* __restrict__ blk, const int64_t* __restrict__ soff,
                                                        int b0, int nb, const RcNode* __restrict__ rows,
                                                        const RcNode* __restrict__ cols,
                                                        const int32_t* __restrict__ rank_r,
                                                        const int32_t* __restrict__ rank_c, unsigned char* arena,
                                                        const double* __restrict__ pool, double* __restrict__ temp) {
    const int b = b0 + blockIdx.x;
    if (b >= nb) return;
    const int t = blk[b].x, s = blk[b].y;
    double* S = reinterpret_cast<double*>(arena + soff[b]);
    const int qt = rows[t].q, qs = cols[s].q, kt = rank_r[t], ks = rank_c[s];
    double* T = temp + (size_t)blockIdx.x * H2_MAX_K * H2_MAX_K;
    cta_gemm(T, qt, S, qt, false, pool + cols[s].B, qs, true, qt, ks, qs);   // S' B_s^T
    __syncthreads();
    cta_gemm(S, kt, pool + rows[t].B, qt, false, T, qt, false, kt, ks, qt);  // B_t (S' B_s^T)
}

}  // namespace

int recompress_device(h2_handle* op, cudaStream_t s) {
    const int nc = op->nc, k = op->k;
    const double eps = op->params.recompress_eps;
    const size_t nfar = op->far_t.size();
    // 0. the interpolation far field in FP64 (leaf bases, transfers as E_c,
    //    couplings) in a scratch arena of its own
    const h2_params saved = op->params;
    op->params.precision = H2_FP64;
    op->params.coupling = H2_COUPLING_STORED;
    op->V.assign(nc, MatRef{});
    op->W.assign(nc, MatRef{});
    op->Eup.assign(nc, MatRef{});
    op->Edown.assign(nc, MatRef{});
    op->S.assign(nfar, MatRef{});
    op->Nb.assign(op->near_t.size(), MatRef{});
    int64_t bytes = 0;
    auto take = [&](MatRef& r, int rows, int cols) {
        r.off = bytes;
        r.nrows = rows;
        r.ncols = cols;
        r.type = PIECE_F64;
        bytes += ((int64_t)rows * cols * 8 + 255) / 256 * 256;
    };
    for (int c = 0; c < nc; ++c) {
        if (op->child0[c] < 0) {
            take(op->V[c], op->size[c], k);   // |c| x k
            take(op->W[c], k, op->size[c]);   // k x |c| (W_c transposed)
        }
        if (op->parent[c] >= 0) take(op->Edown[c], k, k);   // E_c: child x parent
    }
    for (size_t b = 0; b < nfar; ++b) take(op->S[b], k, k);
    auto rcr = new RcResult();
    H2_CUDA_TRY(cudaMalloc((void**)&rcr->d_interp, (size_t)std::max<int64_t>(bytes, 256)));
    unsigned char* interp = reinterpret_cast<unsigned char*>(rcr->d_interp);
    int rc = assemble_interp_far(op, s, interp);
    op->params = saved;
    if (rc != H2_OK) {
        delete rcr;
        return rc;
    }

    // 1. per side, the clusters' descriptors and the pool layout
    int nlev = 0;
    for (int c = 0; c < nc; ++c) nlev = std::max(nlev, op->level[c] + 1);
    std::vector<std::vector<int32_t>> bylev(nlev);
    for (int c = 0; c < nc; ++c) bylev[op->level[c]].push_back(c);
    std::vector<RcNode> nodes[2];
    std::vector<int32_t> blist[2];
    int64_t pool = 0;
    auto grab = [&](int64_t n) {
        const int64_t o = pool;
        pool += (n + 31) / 32 * 32;
        return o;
    };
    for (int side = 0; side < 2; ++side) {
        std::vector<RcNode>& N = nodes[side];
        N.assign(nc, RcNode{});
        std::vector<std::vector<int32_t>> mine(nc);
        for (size_t b = 0; b < nfar; ++b) mine[side == 0 ? op->far_t[b] : op->far_s[b]].push_back((int32_t)b);
        for (int l = nlev - 1; l >= 0; --l)
            for (int c : bylev[l]) {
                RcNode& n = N[c];
                n.leaf = op->child0[c] < 0;
                n.size = op->size[c];
                n.child0 = op->child0[c];
                n.child1 = op->child1[c];
                n.parent = op->parent[c];
                n.second = n.parent >= 0 && op->child1[n.parent] == c;
                n.in = n.leaf ? (side == 0 ? op->V[c].off : op->W[c].off) : -1;
                n.E = n.parent >= 0 ? op->Edown[c].off : -1;
                n.qa = n.leaf ? 0 : N[n.child0].q;
                n.qb = n.leaf ? 0 : N[n.child1].q;
                const int m = n.leaf ? n.size : n.qa + n.qb;
                n.q = std::min(m, k);
                n.blk0 = (int32_t)blist[side].size();
                n.nblk = (int32_t)mine[c].size();
                blist[side].insert(blist[side].end(), mine[c].begin(), mine[c].end());
                const int q = n.q;
                n.R = grab((int64_t)q * k);
                n.Q = grab((int64_t)m * q);
                n.Z = grab((int64_t)q * q);
                n.B = grab((int64_t)q * q);
                n.N = grab((int64_t)m * q);
                // work: the stacked QR input, a condensation, the truncation's G and U (and a leaf's X)
                const int64_t w = std::max({(int64_t)m * k, (int64_t)(q + k) * q, (int64_t)k * q,
                                            (int64_t)3 * m * q});
                n.work = grab(w);
            }
    }
    H2_CUDA_TRY(cudaMalloc((void**)&rcr->d_pool, sizeof(double) * (size_t)std::max<int64_t>(pool, 32)));
    // device copies of the tables
    std::vector<void*> tmp;
    auto cleanup = [&]() {
        for (void* p : tmp) cudaFree(p);
    };
    auto up = [&](const void* h, size_t nbytes, void** d) -> int {
        H2_CUDA_TRY(cudaMalloc(d, std::max<size_t>(nbytes, 16)));
        tmp.push_back(*d);
        if (nbytes) H2_CUDA_TRY(cudaMemcpyAsync(*d, h, nbytes, cudaMemcpyHostToDevice, s));
        return H2_OK;
    };
    RcNode* d_nodes[2];
    int32_t *d_blist[2], *d_zc[2], *d_rank[2];
    std::vector<int2> blk(nfar);
    std::vector<int64_t> soff(nfar);
    for (size_t b = 0; b < nfar; ++b) {
        blk[b] = make_int2(op->far_t[b], op->far_s[b]);
        soff[b] = op->S[b].off;
    }
    int2* d_blk;
    int64_t* d_soff;
    int32_t* d_lev;
    std::vector<int32_t> levall;
    std::vector<int> lev0(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) {
        lev0[l] = (int)levall.size();
        levall.insert(levall.end(), bylev[l].begin(), bylev[l].end());
    }
    lev0[nlev] = (int)levall.size();
    do {
        if ((rc = up(blk.data(), sizeof(int2) * nfar, (void**)&d_blk)) ||
            (rc = up(soff.data(), sizeof(int64_t) * nfar, (void**)&d_soff)) ||
            (rc = up(levall.data(), sizeof(int32_t) * levall.size(), (void**)&d_lev)))
            break;
        const std::vector<int32_t> zeros((size_t)nc, 0);
        for (int side = 0; side < 2 && rc == H2_OK; ++side) {
            if ((rc = up(nodes[side].data(), sizeof(RcNode) * nc, (void**)&d_nodes[side])) ||
                (rc = up(blist[side].data(), sizeof(int32_t) * blist[side].size(), (void**)&d_blist[side])) ||
                (rc = up(zeros.data(), sizeof(int32_t) * nc, (void**)&d_zc[side])) ||
                (rc = up(zeros.data(), sizeof(int32_t) * nc, (void**)&d_rank[side])))
                break;
        }
    } while (false);
    if (rc != H2_OK) {
        cleanup();
        delete rcr;
        return rc;
    }
    // 2. the steps, level by level, on `s`
    cudaError_t e = cudaSuccess;
    auto level_launch = [&](int l, auto&& fn) {
        const int n = lev0[l + 1] - lev0[l];
        if (n > 0) fn(d_lev + lev0[l], n);
    };
    for (int side = 0; side < 2; ++side)   // orthogonalisation, leaves to root
        for (int l = nlev - 1; l >= 0; --l)
            level_launch(l, [&](const int32_t* list, int n) {
                k_rc_orth<<<n, kLaThreads, 0, s>>>(d_nodes[side], list, side, interp, rcr->d_pool, k);
            });
    const int batch = 4096;
    double* d_temp = nullptr;
    if ((e = cudaGetLastError()) == cudaSuccess)
        e = cudaMalloc((void**)&d_temp, sizeof(double) * (size_t)batch * H2_MAX_K * H2_MAX_K);
    if (e == cudaSuccess) {
        tmp.push_back(d_temp);
        for (size_t b0 = 0; b0 < nfar; b0 += batch)   // S' = R_t S R_s^T
            k_rc_sprime<<<(unsigned)std::min<size_t>(batch, nfar - b0), kLaThreads, 0, s>>>(
                d_blk, d_soff, (int)b0, (int)nfar, d_nodes[0], d_nodes[1], interp, rcr->d_pool, d_temp, k);
        for (int side = 0; side < 2; ++side)   // total weights, root to leaves
            for (int l = 0; l < nlev; ++l)
                level_launch(l, [&](const int32_t* list, int n) {
                    k_rc_weights<<<n, kLaThreads, 0, s>>>(d_nodes[side], d_nodes[1 - side], list, side, d_blist[side],
                                                          d_blk, d_soff, interp, rcr->d_pool, d_zc[side]);
                });
        for (int side = 0; side < 2; ++side)   // truncation, leaves to root
            for (int l = nlev - 1; l >= 0; --l)
                level_launch(l, [&](const int32_t* list, int n) {
                    k_rc_truncate<<<n, kLaThreads, 0, s>>>(d_nodes[side], list, rcr->d_pool, d_zc[side], d_rank[side],
                                                           eps);
                });
        for (size_t b0 = 0; b0 < nfar; b0 += batch)   // S'' = B_t S' B_s^T
            k_rc_snew<<<(unsigned)std::min<size_t>(batch, nfar - b0), kLaThreads, 0, s>>>(
                d_blk, d_soff, (int)b0, (int)nfar, d_nodes[0], d_nodes[1], d_rank[0], d_rank[1], interp, rcr->d_pool,
                d_temp);
        e = cudaGetLastError();
    }
    rcr->kr.assign(nc, 0);
    rcr->kc.assign(nc, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rcr->kr.data(), d_rank[0], sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rcr->kc.data(), d_rank[1], sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) {
        set_cuda_error(e, "recompression kernels", __FILE__, __LINE__);
        delete rcr;
        return e == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA;
    }

    // 3. where the product's matrices lie: leaf bases N (ld |c|); a child's
    //    transfer = its rows of the parent's X (ld rank_c0 + rank_c1);
    //    couplings over the interpolation arena (ld rank_t)
    rcr->Vn.assign(nc, RcSource{});
    rcr->Wn.assign(nc, RcSource{});
    rcr->En.assign(nc, RcSource{});
    rcr->Fn.assign(nc, RcSource{});
    rcr->Sn.assign(nfar, RcSource{});
    for (int side = 0; side < 2; ++side) {
        const std::vector<int32_t>& rk = side == 0 ? rcr->kr : rcr->kc;
        std::vector<RcSource>& leafs = side == 0 ? rcr->Vn : rcr->Wn;
        std::vector<RcSource>& trans = side == 0 ? rcr->En : rcr->Fn;
        for (int c = 0; c < nc; ++c) {
            const RcNode& n = nodes[side][c];
            if (n.leaf) leafs[c] = RcSource{n.N, n.size, n.size, rk[c]};
            if (n.parent >= 0) {
                const RcNode& p = nodes[side][n.parent];
                const int a = rk[p.child0] + rk[p.child1];
                trans[c] = RcSource{p.N + (n.second ? rk[p.child0] : 0), a, rk[c], rk[n.parent]};
            }
        }
    }
    for (size_t b = 0; b < nfar; ++b) {
        const int kt = rcr->kr[op->far_t[b]], ks = rcr->kc[op->far_s[b]];
        rcr->Sn[b] = RcSource{op->S[b].off / 8, kt, kt, ks};
    }
    delete op->rc;
    op->rc = rcr;
    return H2_OK;
}

}  // namespace h2
