// Device-side assembly of the boundary operator M = K + D (arXiv:1811.05731,
// Eq. matrix_definition / Eq. denseMat) in H2 form (Section "H2-Matrix
// Compression").  Everything numeric is computed here in FP64; far-field
// matrices are rounded to FP32 on store when the operator is built in FP32.
//
//   k_psi        interior solid angle Psi_i at every node (Eq. mainInt)
//   k_leaf_V     V_t(i, nu)  = L^t_nu(xi_i)                     (row basis)
//   k_leaf_W     W_s(j, mu)  = oint phi_j n . grad L^s_mu dS    (column basis)
//   k_transfer   E_c(nu', nu) = L^parent_nu(x^c_nu')            (nested bases)
//   k_coupling   S_ts(nu, mu) = 1 / (4 pi |x^t_nu - x^s_mu|)
//   k_near       K_ij (Lindholm's closed form) + D_ii on inadmissible leaf pairs
//
// Sign convention of the double-layer term: K_ij = (1/4pi) oint phi_j(y)
// n_y . (xi_i - y) / |xi_i - y|^3 dS_y, under which a constant u1 gives
// u2 = -u1 (the row sums of M are -1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "h2_internal.h"

namespace h2 {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct d3 {
    double x, y, z;
};
__device__ __forceinline__ d3 mk(const double* p) { return {p[0], p[1], p[2]}; }
__device__ __forceinline__ d3 operator-(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ d3 operator*(double s, d3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 cross(d3 a, d3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm(d3 a) { return sqrt(dot(a, a)); }

// ---------------------------------------------------------------------------
// Psi_i: interior solid angle of the surface at node i.  For a closed,
// embedded polyhedral surface the solid angle that all other triangles
// subtend at a node equals the area of the spherical polygon cut out of the
// unit sphere around the node by its fan of triangles.  With the link
// directions u_a (unit vectors to the rim nodes, in the cyclic order given by
// the outward-oriented triangles (i, a, b)), Gauss-Bonnet gives the area on
// the exterior side as 2 pi - sum of turning angles, so the interior angle is
//     Psi_i = 2 pi + sum_b theta_b,
//     theta_b = atan2(det(N1, N2, u_b), N1 . N2),  N1 = u_a x u_b, N2 = u_b x u_c,
// for consecutive rim nodes a -> b -> c.  (A flat node gives 2 pi, a cube
// corner pi / 2.)
// ---------------------------------------------------------------------------
__global__ void k_psi(int64_t N, const double* __restrict__ xyz, const int32_t* __restrict__ tri,
                      const int64_t* __restrict__ adj_ptr, const int32_t* __restrict__ adj,
                      double* __restrict__ psi) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const d3 xi = mk(xyz + 3 * i);
    const int64_t p0 = adj_ptr[i], p1 = adj_ptr[i + 1];
    double sum = 0.0;
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t* v = tri + 3 * (int64_t)adj[p];
        const int c = v[0] == i ? 0 : (v[1] == i ? 1 : 2);
        const int32_t a = v[(c + 1) % 3], b = v[(c + 2) % 3];
        int32_t cnext = -1;
        for (int64_t q = p0; q < p1; ++q) {
            const int32_t* w = tri + 3 * (int64_t)adj[q];
            const int cc = w[0] == i ? 0 : (w[1] == i ? 1 : 2);
            if (w[(cc + 1) % 3] == b) { cnext = w[(cc + 2) % 3]; break; }
        }
        if (cnext < 0) continue;   // rejected by the host-side mesh check
        d3 ua = mk(xyz + 3 * (int64_t)a) - xi, ub = mk(xyz + 3 * (int64_t)b) - xi,
           uc = mk(xyz + 3 * (int64_t)cnext) - xi;
        ua = (1.0 / norm(ua)) * ua;
        ub = (1.0 / norm(ub)) * ub;
        uc = (1.0 / norm(uc)) * uc;
        const d3 n1 = cross(ua, ub), n2 = cross(ub, uc);
        sum += atan2(dot(cross(n1, n2), ub), dot(n1, n2));
    }
    psi[i] = 2.0 * kPi + sum;
}

// ---------------------------------------------------------------------------
// Chebyshev interpolation on an axis-parallel box: m points of the first kind
// per axis, c + (w/2) cos((2j+1) pi / (2m)), tensor index nu = (a m + b) m + c.
// ---------------------------------------------------------------------------
struct Cheb {
    double p[3][H2_MAX_M];
};

__device__ __forceinline__ void cheb_nodes(const double* box, int m, Cheb& cb) {
    for (int d = 0; d < 3; ++d) {
        const double c = 0.5 * (box[d] + box[3 + d]), h = 0.5 * (box[3 + d] - box[d]);
        for (int j = 0; j < m; ++j) cb.p[d][j] = c + h * cos((2.0 * j + 1.0) * kPi / (2.0 * m));
    }
}

// Lagrange polynomial of node j among p[0..m-1] at t.
__device__ __forceinline__ double lagr(const double* p, int m, int j, double t) {
    double v = 1.0;
    for (int l = 0; l < m; ++l)
        if (l != j) v *= (t - p[l]) / (p[j] - p[l]);
    return v;
}
// Its derivative: sum over the dropped factor q of the remaining product.
__device__ __forceinline__ double dlagr(const double* p, int m, int j, double t) {
    double s = 0.0;
    for (int q = 0; q < m; ++q) {
        if (q == j) continue;
        double v = 1.0 / (p[j] - p[q]);
        for (int l = 0; l < m; ++l)
            if (l != j && l != q) v *= (t - p[l]) / (p[j] - p[l]);
        s += v;
    }
    return s;
}

__device__ __forceinline__ void store(unsigned char* arena, int64_t off, int64_t idx, double v,
                                      int f32) {
    if (f32) reinterpret_cast<float*>(arena + off)[idx] = (float)v;
    else reinterpret_cast<double*>(arena + off)[idx] = v;
}

// Stores entry (i, j) of an nrows-row far-field block in the operator's
// format `type` (a PieceType): column-major FP64 / FP32, a TF32 tensor tile
// (FP32 values), or a BF16 hi + lo tensor tile (hi = bf16(v), lo = bf16(v - hi)).
__device__ __forceinline__ void store_block(unsigned char* arena, int64_t off, int nrows, int i, int j, double v,
                                            int type) {
    if (type == PIECE_F64) {
        reinterpret_cast<double*>(arena + off)[(int64_t)j * nrows + i] = v;
    } else if (type == PIECE_F32) {
        reinterpret_cast<float*>(arena + off)[(int64_t)j * nrows + i] = (float)v;
    } else if (type == PIECE_TF32) {
        *reinterpret_cast<float*>(arena + off + tc_offset(type, tc_rows(nrows), i, j, 0)) = (float)v;
    } else {
        const __nv_bfloat16 hi = __double2bfloat16(v);
        const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16*>(arena + off + tc_offset(type, tc_rows(nrows), i, j, 0)) = hi;
        *reinterpret_cast<__nv_bfloat16*>(arena + off + tc_offset(type, tc_rows(nrows), i, j, 1)) = lo;
    }
}

struct BasisItem {
    double box[6];
    int64_t off;
    int32_t start, size;
};

// V_t (|t| x k, column-major: (a, nu) at nu*|t| + a).
__global__ void k_leaf_V(const BasisItem* __restrict__ items, int m, const int32_t* __restrict__ perm,
                         const double* __restrict__ xyz, unsigned char* arena, int f32) {
    const BasisItem it = items[blockIdx.x];
    const int k = m * m * m;
    const int nu = threadIdx.x;
    if (nu >= k) return;
    Cheb cb;
    cheb_nodes(it.box, m, cb);
    const int a = nu / (m * m), b = (nu / m) % m, c = nu % m;
    for (int q = 0; q < it.size; ++q) {
        const double* x = xyz + 3 * (int64_t)perm[it.start + q];
        const double v = lagr(cb.p[0], m, a, x[0]) * lagr(cb.p[1], m, b, x[1]) *
                         lagr(cb.p[2], m, c, x[2]);
        store(arena, it.off, (int64_t)nu * it.size + q, v, f32);
    }
}

struct LeafTri {
    int32_t tri;
    int32_t col[3];     // column of each corner in the source leaf, -1 outside
};

struct WItem {
    double box[6];
    int64_t off;
    int32_t size;       // nodes of the leaf
    int32_t tl0, tl1;   // its triangles in the leaf-triangle list
};

// W_s (k x |s| column-major: (mu, j) at j*k + mu), the integral of phi_j
// n . grad L_mu over the triangles around node j, by a collapsed (Duffy)
// Gauss-Legendre product rule with q points per direction, exact for the
// polynomial integrand of total degree 3(m-1) when 2q - 1 >= 3m - 2.
// One CTA per leaf; the leaf's triangles are visited once and every Gauss
// point contributes to the corners of the triangle that belong to the leaf.
// Thread mu owns column mu of the leaf's block in shared memory.  At a point
// y, lane l < 3m of each warp evaluates the Lagrange factor L_{d,j}(y_d)
// (d = l / m, j = l % m) and lane 3m + l its derivative, in product form with
// barycentric weights (no divisions), and the threads gather the six factors
// of L_mu and grad L_mu by shuffles.
__global__ void k_leaf_W(const WItem* __restrict__ items, const LeafTri* __restrict__ ltri, int m,
                         const double* __restrict__ xyz, const int32_t* __restrict__ tri,
                         const double* __restrict__ gx, const double* __restrict__ gw, int q,
                         unsigned char* arena, int f32) {
    extern __shared__ double wsm[];
    const WItem it = items[blockIdx.x];
    const int k = m * m * m;
    const int mu = threadIdx.x;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < it.size * k; i += blockDim.x) wsm[i] = 0.0;
    Cheb cb;
    cheb_nodes(it.box, m, cb);
    double wbar[3][H2_MAX_M];
    for (int d = 0; d < 3; ++d)
        for (int j = 0; j < m; ++j) {
            double v = 1.0;
            for (int l = 0; l < m; ++l)
                if (l != j) v *= cb.p[d][j] - cb.p[d][l];
            wbar[d][j] = 1.0 / v;
        }
    // this lane's factor: value (role < 3m) or derivative (3m <= role < 6m)
    const int role = lane < 6 * m ? lane : -1;
    const int fd = role >= 0 ? (role % (3 * m)) / m : 0;
    const int fj = role >= 0 ? role % m : 0;
    const bool fder = role >= 3 * m;
    const int a = mu / (m * m), b = (mu / m) % m, c = mu % m;
    __syncthreads();
    for (int t = it.tl0; t < it.tl1; ++t) {
        const LeafTri lt = ltri[t];
        const int32_t* v = tri + 3 * (int64_t)lt.tri;
        const d3 r0 = mk(xyz + 3 * (int64_t)v[0]), r1 = mk(xyz + 3 * (int64_t)v[1]),
                 r2 = mk(xyz + 3 * (int64_t)v[2]);
        const d3 e1 = r1 - r0, e2 = r2 - r0;
        const d3 nn = cross(e1, e2);
        const double twoA = norm(nn);
        const d3 n = (1.0 / twoA) * nn;
        for (int iu = 0; iu < q; ++iu) {
            const double sc = gx[iu];
            for (int iv = 0; iv < q; ++iv) {
                const double tc = gx[iv] * (1.0 - sc);
                const double wt = gw[iu] * gw[iv] * (1.0 - sc) * twoA;
                const d3 y = r0 + (sc * e1 + tc * e2);
                double f = 0.0;
                if (role >= 0) {
                    const double x = fd == 0 ? y.x : (fd == 1 ? y.y : y.z);
                    const double* p = cb.p[fd];
                    if (!fder) {
                        f = 1.0;
                        for (int l = 0; l < m; ++l)
                            if (l != fj) f *= x - p[l];
                    } else {
                        for (int q2 = 0; q2 < m; ++q2) {
                            if (q2 == fj) continue;
                            double pr = 1.0;
                            for (int l = 0; l < m; ++l)
                                if (l != fj && l != q2) pr *= x - p[l];
                            f += pr;
                        }
                    }
                    f *= wbar[fd][fj];
                }
                const double lx = __shfl_sync(~0u, f, a), ly = __shfl_sync(~0u, f, m + b),
                             lz = __shfl_sync(~0u, f, 2 * m + c), dx = __shfl_sync(~0u, f, 3 * m + a),
                             dy = __shfl_sync(~0u, f, 4 * m + b), dz = __shfl_sync(~0u, f, 5 * m + c);
                if (mu < k) {
                    const double g = n.x * dx * ly * lz + n.y * lx * dy * lz + n.z * lx * ly * dz;
                    const double wg = wt * g;
                    if (lt.col[0] >= 0) wsm[lt.col[0] * k + mu] += wg * (1.0 - sc - tc);
                    if (lt.col[1] >= 0) wsm[lt.col[1] * k + mu] += wg * sc;
                    if (lt.col[2] >= 0) wsm[lt.col[2] * k + mu] += wg * tc;
                }
            }
        }
    }
    if (mu < k)
        for (int j = 0; j < it.size; ++j) store(arena, it.off, (int64_t)j * k + mu, wsm[j * k + mu], f32);
}

struct TransferItem {
    double box_child[6], box_parent[6];
    int64_t off_up, off_down;   // -1 when not stored
};

// E_c(nu', nu) = L^parent_nu(x^c_nu').  Up layout (nu, nu') at nu'*k + nu,
// down layout (nu', nu) at nu*k + nu'.
__global__ void k_transfer(const TransferItem* __restrict__ items, int m, unsigned char* arena,
                           int type) {
    const TransferItem& it = items[blockIdx.x];
    const int k = m * m * m;
    const int nu = threadIdx.x;
    if (nu >= k) return;
    Cheb cc, cp;
    cheb_nodes(it.box_child, m, cc);
    cheb_nodes(it.box_parent, m, cp);
    const int a = nu / (m * m), b = (nu / m) % m, c = nu % m;
    for (int np = 0; np < k; ++np) {
        const int a2 = np / (m * m), b2 = (np / m) % m, c2 = np % m;
        const double v = lagr(cp.p[0], m, a, cc.p[0][a2]) * lagr(cp.p[1], m, b, cc.p[1][b2]) *
                         lagr(cp.p[2], m, c, cc.p[2][c2]);
        if (it.off_up >= 0) store_block(arena, it.off_up, k, nu, np, v, type);
        if (it.off_down >= 0) store_block(arena, it.off_down, k, np, nu, v, type);
    }
}

struct CouplingItem {
    int32_t t, s;
    int64_t off;
};

// S_ts (k x k column-major: (nu, mu) at mu*k + nu).
__global__ void k_coupling(const CouplingItem* __restrict__ items, int m,
                           const double* __restrict__ box, unsigned char* arena, int type) {
    const CouplingItem it = items[blockIdx.x];
    const int k = m * m * m;
    __shared__ double pt[3][H2_MAX_K], ps[3][H2_MAX_K];
    __shared__ Cheb ct, cs;
    if (threadIdx.x == 0) {
        cheb_nodes(box + 6 * (int64_t)it.t, m, ct);
        cheb_nodes(box + 6 * (int64_t)it.s, m, cs);
    }
    __syncthreads();
    for (int nu = threadIdx.x; nu < k; nu += blockDim.x) {
        const int a = nu / (m * m), b = (nu / m) % m, c = nu % m;
        pt[0][nu] = ct.p[0][a]; pt[1][nu] = ct.p[1][b]; pt[2][nu] = ct.p[2][c];
        ps[0][nu] = cs.p[0][a]; ps[1][nu] = cs.p[1][b]; ps[2][nu] = cs.p[2][c];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        const int mu = idx / k, nu = idx % k;
        const double dx = pt[0][nu] - ps[0][mu], dy = pt[1][nu] - ps[1][mu],
                     dz = pt[2][nu] - ps[2][mu];
        const double v = 1.0 / (4.0 * kPi * sqrt(dx * dx + dy * dy + dz * dz));
        store_block(arena, it.off, k, nu, mu, v, type);
    }
}

// Coupling blocks evaluated in the product (H2_COUPLING_ON_THE_FLY): per block,
// the source cluster's Chebyshev nodes minus the target box's centre, one
// float4 per column (the difference in FP64, rounded once).
__global__ void k_coupling_nodes(const CouplingItem* __restrict__ items, int m, const double* __restrict__ box,
                                 unsigned char* arena) {
    const CouplingItem it = items[blockIdx.x];
    const int k = m * m * m;
    __shared__ double off[3], h[3], cosv[H2_MAX_M];
    if (threadIdx.x == 0) {
        for (int d = 0; d < 3; ++d) {
            const double* bs = box + 6 * (int64_t)it.s;
            const double* bt = box + 6 * (int64_t)it.t;
            off[d] = 0.5 * (bs[d] + bs[3 + d]) - 0.5 * (bt[d] + bt[3 + d]);   // source centre - target centre
            h[d] = 0.5 * (bs[3 + d] - bs[d]);
        }
        for (int j = 0; j < m; ++j) cosv[j] = cos((2.0 * j + 1.0) * kPi / (2.0 * m));
    }
    __syncthreads();
    float4* dst = reinterpret_cast<float4*>(arena + it.off);
    for (int mu = threadIdx.x; mu < k; mu += blockDim.x) {
        const int a = mu / (m * m), b = (mu / m) % m, c = mu % m;
        dst[mu] = make_float4((float)(off[0] + h[0] * cosv[a]), (float)(off[1] + h[1] * cosv[b]),
                              (float)(off[2] + h[2] * cosv[c]), 0.0f);
    }
}

// Every cluster's Chebyshev nodes minus its box's centre (kp float4 per
// cluster): the target side of the evaluated coupling blocks.
__global__ void k_cluster_nodes(int m, int kp, const double* __restrict__ box, float4* __restrict__ out) {
    const int cl = blockIdx.x;
    const int k = m * m * m;
    const double* b = box + 6 * (int64_t)cl;
    for (int nu = threadIdx.x; nu < kp; nu += blockDim.x) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (nu < k) {
            const int ia[3] = {nu / (m * m), (nu / m) % m, nu % m};
            float w[3];
            for (int d = 0; d < 3; ++d)
                w[d] = (float)(0.5 * (b[3 + d] - b[d]) * cos((2.0 * ia[d] + 1.0) * kPi / (2.0 * m)));
            v = make_float4(w[0], w[1], w[2], 0.0f);
        }
        out[(int64_t)cl * kp + nu] = v;
    }
}

// ---------------------------------------------------------------------------
// Lindholm's closed form for a linear basis on a flat triangle.  For the
// triangle T = (r0, r1, r2) with unit normal n ~ (r1 - r0) x (r2 - r0), area A,
// edge b from r_b to r_{b+1} (length s_b, direction sh_b) and the observation
// point x (rho_b = r_b - x, R_b = |rho_b|, zeta = n . rho_0):
//   P_b     = ln((R_b + R_{b+1} + s_b) / (R_b + R_{b+1} - s_b))
//   eta_b   = (n x sh_b) . rho_b
//   Omega   = solid angle of T at x (Van Oosterom-Strackee)
//   w_a     = s_{a+1} / (8 pi A) [ eta_{a+1} Omega - zeta sum_b (sh_{a+1} . sh_b) P_b ]
// where w_a = (1/4pi) int_T phi_a n . (x - y) / |x - y|^3 dS_y.  A point in the
// plane of T (|zeta| <= 1e-13 sqrt(A)) sees no double-layer contribution.
// ---------------------------------------------------------------------------
__device__ void lindholm_weights(d3 x, d3 r0, d3 r1, d3 r2, double w[3]) {
    const d3 r[3] = {r0, r1, r2};
    d3 rho[3], sh[3];
    double R[3], sl[3];
    for (int b = 0; b < 3; ++b) {
        rho[b] = r[b] - x;
        R[b] = norm(rho[b]);
        const d3 e = r[(b + 1) % 3] - r[b];
        sl[b] = norm(e);
        sh[b] = (1.0 / sl[b]) * e;
    }
    const d3 nn = cross(r1 - r0, r2 - r0);
    const double twoA = norm(nn);
    const double A = 0.5 * twoA;
    const d3 n = (1.0 / twoA) * nn;
    const double zeta = dot(n, rho[0]);
    if (fabs(zeta) <= 1e-13 * sqrt(A)) {
        w[0] = w[1] = w[2] = 0.0;
        return;
    }
    const double num = dot(rho[0], cross(rho[1], rho[2]));
    const double den = R[0] * R[1] * R[2] + dot(rho[0], rho[1]) * R[2] +
                       dot(rho[0], rho[2]) * R[1] + dot(rho[1], rho[2]) * R[0];
    const double omega = 2.0 * atan2(num, den);
    double P[3], eta[3];
    for (int b = 0; b < 3; ++b) {
        const double Rs = R[b] + R[(b + 1) % 3];
        P[b] = log((Rs + sl[b]) / (Rs - sl[b]));
        eta[b] = dot(cross(n, sh[b]), rho[b]);
    }
    const double pre = 1.0 / (8.0 * kPi * A);
    for (int a = 0; a < 3; ++a) {
        const int o = (a + 1) % 3;
        const double g = dot(sh[o], sh[0]) * P[0] + dot(sh[o], sh[1]) * P[1] +
                         dot(sh[o], sh[2]) * P[2];
        w[a] = sl[o] * pre * (eta[o] * omega - zeta * g);
    }
}

struct NearItem {
    int64_t off;
    int32_t t_start, t_size, s_start, s_size;
    int32_t tl0, tl1;   // range in the source leaf's triangle list
    int32_t diag;       // t == s
    int32_t pad;
};

// One near block N_ts (|t| x |s| column-major: (a, b) at b*|t| + a) per CTA;
// thread a owns row a and sums the corner weights of every triangle around
// the source leaf into the columns of the corners that belong to s.
// The paired copy of the near blocks (h2_near_field H2_NEAR_F32PAIR): every
// FP64 value v of the near pass's arena bytes as hi = fp32(v) and
// lo = fp32(v - hi), the exact remainder rounded once (48 significant bits).
// One recompressed far-field matrix: an FP64 column-major source (rows x
// cols, leading dimension ld) copied, transposed when `trans`, into an
// arena block of `nrows` rows in the product's format `type`.
struct StoreItem {
    int64_t src;        // doubles into the source buffer
    int64_t dst;        // bytes into the arena
    int32_t ld, rows, cols, trans, nrows, type;
};

__global__ void k_store_rc(const StoreItem* __restrict__ items, const double* __restrict__ src0,
                           const double* __restrict__ src1, unsigned char* arena) {
    const StoreItem it = items[blockIdx.x];
    const double* src = it.trans < 2 ? src0 : src1;   // trans bit 1: the second source buffer
    const bool tr = (it.trans & 1) != 0;
    const int orow = tr ? it.cols : it.rows, ocol = tr ? it.rows : it.cols;
    for (int idx = threadIdx.x; idx < orow * ocol; idx += blockDim.x) {
        const int i = idx % orow, j = idx / orow;
        const double v = tr ? src[it.src + (int64_t)i * it.ld + j] : src[it.src + (int64_t)j * it.ld + i];
        store_block(arena, it.dst, it.nrows, i, j, v, it.type);
    }
}

__global__ void k_pair_split(const double* __restrict__ src, float2* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = src[i];
        const float hi = __double2float_rn(v);
        dst[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

__global__ void k_near(const NearItem* __restrict__ items, const LeafTri* __restrict__ ltri,
                       const int32_t* __restrict__ perm, const double* __restrict__ xyz,
                       const int32_t* __restrict__ tri, const double* __restrict__ psi,
                       unsigned char* arena) {
    extern __shared__ double blk[];
    const NearItem it = items[blockIdx.x];
    const int nt = it.t_size, ns = it.s_size;
    for (int idx = threadIdx.x; idx < nt * ns; idx += blockDim.x) blk[idx] = 0.0;
    __syncthreads();
    const int a = threadIdx.x;
    if (a < nt) {
        const int32_t i = perm[it.t_start + a];
        const d3 x = mk(xyz + 3 * (int64_t)i);
        for (int e = it.tl0; e < it.tl1; ++e) {
            const LeafTri lt = ltri[e];
            const int32_t* v = tri + 3 * (int64_t)lt.tri;
            if (v[0] == i || v[1] == i || v[2] == i) continue;
            double w[3];
            lindholm_weights(x, mk(xyz + 3 * (int64_t)v[0]), mk(xyz + 3 * (int64_t)v[1]),
                             mk(xyz + 3 * (int64_t)v[2]), w);
            for (int q = 0; q < 3; ++q)
                if (lt.col[q] >= 0) blk[lt.col[q] * nt + a] += w[q];
        }
        if (it.diag) blk[a * nt + a] += psi[i] / (4.0 * kPi) - 1.0;
    }
    __syncthreads();
    double* out = reinterpret_cast<double*>(arena + it.off);
    for (int idx = threadIdx.x; idx < nt * ns; idx += blockDim.x) out[idx] = blk[idx];
}

template <class Tv>
int upload(const std::vector<Tv>& v, Tv** d, cudaStream_t s) {
    *d = nullptr;
    if (v.empty()) return H2_OK;
    H2_CUDA_TRY(cudaMalloc((void**)d, sizeof(Tv) * v.size()));
    H2_CUDA_TRY(cudaMemcpyAsync(*d, v.data(), sizeof(Tv) * v.size(), cudaMemcpyHostToDevice, s));
    return H2_OK;
}

}  // namespace

int geometry_device_setup(h2_handle* g, cudaStream_t s) {
    int rc;
    if ((rc = upload(g->xyz, &g->d_xyz, s))) return rc;
    if ((rc = upload(g->tri, &g->d_tri, s))) return rc;
    if ((rc = upload(g->adj_ptr, &g->d_adj_ptr, s))) return rc;
    if ((rc = upload(g->adj, &g->d_adj, s))) return rc;
    H2_CUDA_TRY(cudaMalloc((void**)&g->d_psi, sizeof(double) * g->N));
    const int bs = 128;
    k_psi<<<(unsigned)((g->N + bs - 1) / bs), bs, 0, s>>>(g->N, g->d_xyz, g->d_tri, g->d_adj_ptr,
                                                          g->d_adj, g->d_psi);
    H2_CUDA_TRY(cudaGetLastError());
    H2_CUDA_TRY(cudaStreamSynchronize(s));
    return H2_OK;
}

// Assembles the operator's matrices into `arena` at the offsets its plan
// recorded (h2_handle::V, W, Eup, Edown, S, Nb): the interpolation far field
// (leaf bases, transfers, couplings) when `far`, the near blocks when `near`.
static int assemble_matrices(h2_handle* op, cudaStream_t s, unsigned char* arena, bool far, bool near) {
    const h2_handle* g = op->geom;
    const int m = op->m, k = op->k;
    // leaf bases: FP64 or FP32 column-major; coupling and transfer blocks in
    // the operator's far-field format
    const int prec = op->params.precision;
    const int f32 = prec == H2_FP64 ? 0 : 1;
    const int tt = coupling_piece_type(prec);    // coupling blocks
    const int te = transfer_piece_type(prec);    // transfers
    int rc;

    if (!op->d_perm && (rc = upload(op->perm, &op->d_perm, s))) return rc;
    if (!op->d_box && (rc = upload(op->box, &op->d_box, s))) return rc;

    std::vector<void*> tmp;
    auto cleanup = [&]() {
        for (void* p : tmp) cudaFree(p);
        tmp.clear();
    };

    // leaf bases
    std::vector<BasisItem> vi;
    for (int c = 0; c < op->nc; ++c) {
        BasisItem it{};
        std::memcpy(it.box, &op->box[6 * (size_t)c], sizeof(it.box));
        it.start = op->start[c];
        it.size = op->size[c];
        if (far && op->V[c].off >= 0) { it.off = op->V[c].off; vi.push_back(it); }
    }
    std::vector<double> gx, gw;
    const int q = (3 * m) / 2;   // ceil((3m - 1) / 2)
    gauss_legendre_unit(q, gx, gw);
    BasisItem* d_vi = nullptr;
    double *d_gx = nullptr, *d_gw = nullptr;
    if ((rc = upload(vi, &d_vi, s)) || (rc = upload(gx, &d_gx, s)) || (rc = upload(gw, &d_gw, s))) {
        cleanup();
        return rc;
    }
    tmp.insert(tmp.end(), {d_vi, d_gx, d_gw});
    const int kb = (k + 31) / 32 * 32;
    if (!vi.empty())
        k_leaf_V<<<(unsigned)vi.size(), kb, 0, s>>>(d_vi, m, op->d_perm, g->d_xyz, arena, f32);

    // per leaf, the triangles around its nodes (column bases and near field)
    std::vector<int32_t> leaf_pos(op->nc, -1);
    std::vector<LeafTri> ltri;
    std::vector<int32_t> ltr0(op->nc, 0), ltr1(op->nc, 0);
    {
        std::vector<int32_t> col_of((size_t)g->N, -1);
        std::vector<int32_t> seen((size_t)g->T, -1);
        for (int c = 0; c < op->nc; ++c) {
            if (op->child0[c] >= 0) continue;
            for (int a = 0; a < op->size[c]; ++a) col_of[op->perm[op->start[c] + a]] = a;
            ltr0[c] = (int32_t)ltri.size();
            for (int a = 0; a < op->size[c]; ++a) {
                const int32_t j = op->perm[op->start[c] + a];
                for (int64_t p = g->adj_ptr[j]; p < g->adj_ptr[j + 1]; ++p) {
                    const int32_t t = g->adj[p];
                    if (seen[t] == c) continue;
                    seen[t] = c;
                    LeafTri lt{};
                    lt.tri = t;
                    for (int q2 = 0; q2 < 3; ++q2) lt.col[q2] = col_of[g->tri[3 * (size_t)t + q2]];
                    ltri.push_back(lt);
                }
            }
            ltr1[c] = (int32_t)ltri.size();
            for (int a = 0; a < op->size[c]; ++a) col_of[op->perm[op->start[c] + a]] = -1;
        }
    }
    LeafTri* d_lt = nullptr;
    if ((rc = upload(ltri, &d_lt, s))) { cleanup(); return rc; }
    tmp.push_back(d_lt);
    {
        std::vector<WItem> wj;
        int maxw = 1;
        for (int c = 0; c < op->nc; ++c) {
            if (!far || op->W[c].off < 0) continue;
            WItem it{};
            std::memcpy(it.box, &op->box[6 * (size_t)c], sizeof(it.box));
            it.off = op->W[c].off;
            it.size = op->size[c];
            it.tl0 = ltr0[c];
            it.tl1 = ltr1[c];
            wj.push_back(it);
            maxw = std::max(maxw, it.size);
        }
        WItem* d_wj = nullptr;
        if ((rc = upload(wj, &d_wj, s))) { cleanup(); return rc; }
        tmp.push_back(d_wj);
        if (!wj.empty()) {
            const size_t smem = sizeof(double) * (size_t)maxw * k;
            H2_CUDA_TRY(cudaFuncSetAttribute(k_leaf_W, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_leaf_W<<<(unsigned)wj.size(), kb, smem, s>>>(d_wj, d_lt, m, g->d_xyz, g->d_tri, d_gx, d_gw, q,
                                                           arena, f32);
        }
    }

    // transfers
    std::vector<TransferItem> ti;
    for (int c = 0; c < op->nc; ++c) {
        if (!far || (op->Eup[c].off < 0 && op->Edown[c].off < 0)) continue;
        TransferItem it{};
        std::memcpy(it.box_child, &op->box[6 * (size_t)c], sizeof(it.box_child));
        std::memcpy(it.box_parent, &op->box[6 * (size_t)op->parent[c]], sizeof(it.box_parent));
        it.off_up = op->Eup[c].off;
        it.off_down = op->Edown[c].off;
        ti.push_back(it);
    }
    TransferItem* d_ti = nullptr;
    if ((rc = upload(ti, &d_ti, s))) { cleanup(); return rc; }
    tmp.push_back(d_ti);
    if (!ti.empty()) k_transfer<<<(unsigned)ti.size(), kb, 0, s>>>(d_ti, m, arena, te);

    // coupling
    std::vector<CouplingItem> ci(far ? op->far_t.size() : 0);
    for (size_t b = 0; b < ci.size(); ++b) ci[b] = {op->far_t[b], op->far_s[b], op->S[b].off};
    CouplingItem* d_ci = nullptr;
    if ((rc = upload(ci, &d_ci, s))) { cleanup(); return rc; }
    tmp.push_back(d_ci);
    if (far && op->params.coupling == H2_COUPLING_ON_THE_FLY) {   // nodes only: the product evaluates S_ts
        if (!op->d_nodes) H2_CUDA_TRY(cudaMalloc((void**)&op->d_nodes, sizeof(float4) * (size_t)op->nc * op->kp));
        k_cluster_nodes<<<(unsigned)op->nc, 128, 0, s>>>(m, op->kp, op->d_box, op->d_nodes);
        if (!ci.empty()) k_coupling_nodes<<<(unsigned)ci.size(), 128, 0, s>>>(d_ci, m, op->d_box, arena);
    } else if (!ci.empty()) {
        k_coupling<<<(unsigned)ci.size(), 256, 0, s>>>(d_ci, m, op->d_box, arena, tt);
    }

    std::vector<NearItem> ni(near ? op->near_t.size() : 0);
    int maxleaf = 1;
    for (size_t b = 0; b < ni.size(); ++b) {
        const int t = op->near_t[b], sc = op->near_s[b];
        NearItem it{};
        it.off = op->Nb[b].off;
        it.t_start = op->start[t];
        it.t_size = op->size[t];
        it.s_start = op->start[sc];
        it.s_size = op->size[sc];
        it.tl0 = ltr0[sc];
        it.tl1 = ltr1[sc];
        it.diag = t == sc;
        ni[b] = it;
        maxleaf = std::max(maxleaf, std::max(it.t_size, it.s_size));
    }
    NearItem* d_ni = nullptr;
    if ((rc = upload(ni, &d_ni, s))) { cleanup(); return rc; }
    tmp.push_back(d_ni);
    if (!ni.empty()) {
        const size_t smem = sizeof(double) * (size_t)maxleaf * maxleaf;
        H2_CUDA_TRY(cudaFuncSetAttribute(k_near, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int nb = (maxleaf + 31) / 32 * 32;
        k_near<<<(unsigned)ni.size(), nb, smem, s>>>(d_ni, d_lt, op->d_perm, g->d_xyz, g->d_tri,
                                                     g->d_psi, arena);
    }
    if (near && op->d_near_pair && op->near_hi > op->near_lo) {
        const int64_t n = (op->near_hi - op->near_lo) / 8;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16 * 152));
        k_pair_split<<<grid, 256, 0, s>>>(reinterpret_cast<const double*>(arena + op->near_lo),
                                          op->d_near_pair, n);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return H2_ERR_CUDA;
    }
    return H2_OK;
}

// The operator's arena: the far field from the recompression when the
// operator was recompressed (h2_params.recompress_eps > 0), else from the
// interpolation kernels; the near blocks always.
int assemble_device(h2_handle* op, cudaStream_t s) {
    H2_CUDA_TRY(cudaMalloc((void**)&op->d_arena, (size_t)std::max<int64_t>(op->arena_bytes, 16)));
    H2_CUDA_TRY(cudaMemsetAsync(op->d_arena, 0, (size_t)std::max<int64_t>(op->arena_bytes, 16), s));
    if (op->rc) {
        const RcResult& R = *op->rc;
        const int prec = op->params.precision;
        const int P = prec == H2_FP64 ? PIECE_F64 : PIECE_F32;
        const int PT = transfer_piece_type(prec), PC = coupling_piece_type(prec);
        std::vector<StoreItem> items;
        auto add = [&](const RcSource& src, const MatRef& dst, int trans, int type, bool second) {
            if (dst.off < 0 || src.rows <= 0 || src.cols <= 0) return;
            items.push_back(StoreItem{src.off, dst.off, src.ld, src.rows, src.cols, trans | (second ? 2 : 0),
                                      dst.nrows, type});
        };
        for (int c = 0; c < op->nc; ++c) {
            // W block: kc x |c| with entry (mu, j) = Wn(j, mu); V block: |c| x kr = Vn
            if (op->child0[c] < 0) {
                add(R.Wn[c], op->W[c], 1, P, false);
                add(R.Vn[c], op->V[c], 0, P, false);
            }
            // upward transfer into the parent: kc_p x kc_c = Fn_c^T; downward: kr_c x kr_p = En_c
            if (op->parent[c] >= 0) {
                add(R.Fn[c], op->Eup[c], 1, PT, false);
                add(R.En[c], op->Edown[c], 0, PT, false);
            }
        }
        for (size_t b = 0; b < op->far_t.size(); ++b) add(R.Sn[b], op->S[b], 0, PC, true);
        StoreItem* d_items = nullptr;
        int rc = upload(items, &d_items, s);
        if (rc) return rc;
        if (!items.empty()) k_store_rc<<<(unsigned)items.size(), 256, 0, s>>>(d_items, R.d_pool, R.d_interp, op->d_arena);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_items);
        if (e != cudaSuccess) {
            set_cuda_error(e, "k_store_rc", __FILE__, __LINE__);
            return H2_ERR_CUDA;
        }
        return assemble_matrices(op, s, op->d_arena, false, true);
    }
    return assemble_matrices(op, s, op->d_arena, true, true);
}

// The interpolation far field alone, in FP64, into `arena` at the offsets
// the caller recorded in the operator's matrix references (recompression input).
int assemble_interp_far(h2_handle* op, cudaStream_t s, unsigned char* arena) {
    return assemble_matrices(op, s, arena, true, false);
}

}  // namespace h2
