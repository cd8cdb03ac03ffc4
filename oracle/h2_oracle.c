/*
 * CPU oracle for the boundary double-layer operator of the Fredkin-Koehler
 * FEM/BEM method and for its interpolation-based H2 approximation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no source with
 * the CUDA path and is never used to produce a product result.
 *
 * Plain, slow, FP64 throughout.  What it computes (section and equation
 * names of arXiv:1811.05731):
 *
 *  - Collocation matrix M = K + D of Eq. (matrix_definition) / Eq. (denseMat):
 *      K_ij = (1/4pi) \oint phi_j(y) n_y.(xi_i - y)/|xi_i - y|^3 dS_y
 *      D_ii = Psi(xi_i)/(4 pi) - 1
 *    (sign of the double-layer term: the reading under which a constant u1
 *    gives u2 = -u1, i.e. M 1 = -1; the paper's printed sign of dG/dn with
 *    G = -1/(4 pi r) would give the opposite sign, Eq. (mainInt)).
 *  - K_ij by the analytic Lindholm formula for a linear basis function on a
 *    flat triangle (the paper cites Lindholm 1984 and does not print it; the
 *    formula is re-derived here from the divergence theorem in the plane).
 *  - Psi_i: interior solid angle at node i, the sum of the Van Oosterom-
 *    Strackee solid angles of all triangles not containing node i (Eq.
 *    (mainInt), "solid angle subtended at x").
 *  - The H2 approximation of Section "H2-Matrix Compression": a geometric
 *    cluster tree, eta-admissible block partition and, for every admissible
 *    block (t, s), K|_{t x s} ~ V_t S_ts W_s^T with tensor Chebyshev
 *    interpolation of g(x, y) = 1/(4 pi |x - y|) on each cluster's box:
 *      V_t(i, nu) = L^t_nu(xi_i)
 *      S_ts(nu, mu) = g(x^t_nu, x^s_mu)
 *      W_s(j, mu) = \oint phi_j(y) n_y . grad L^s_mu(y) dS_y
 *    The oracle evaluates V_t and W_s directly on each cluster's own box (no
 *    transfer matrices), so it is independent of the nested form.
 *
 * Parity unpinned: none (every function here is checked by a test against a
 * value fixed independently of this file).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define O_PI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static inline void vsub(const double* a, const double* b, double* c) {
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
static inline double vdot(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static inline void vcross(const double* a, const double* b, double* c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double vnorm(const double* a) { return sqrt(vdot(a, a)); }

int o_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* solid angle and Lindholm corner weights                            */
/* ------------------------------------------------------------------ */

/* Signed solid angle subtended at x by the oriented triangle (a, b, c):
 * Omega = \int_T n.(y - x)/|y - x|^3 dS, positive when x lies on the side the
 * normal (b-a)x(c-a) points away from.  Van Oosterom & Strackee (1983):
 * tan(Omega/2) = r1.(r2 x r3) / (|r1||r2||r3| + (r1.r2)|r3| + (r1.r3)|r2| + (r2.r3)|r1|). */
double o_solid_angle(const double* x, const double* a, const double* b, const double* c) {
    double r1[3], r2[3], r3[3], cr[3];
    vsub(a, x, r1); vsub(b, x, r2); vsub(c, x, r3);
    double l1 = vnorm(r1), l2 = vnorm(r2), l3 = vnorm(r3);
    vcross(r2, r3, cr);
    double num = vdot(r1, cr);
    double den = l1 * l2 * l3 + vdot(r1, r2) * l3 + vdot(r1, r3) * l2 + vdot(r2, r3) * l1;
    return 2.0 * atan2(num, den);
}

/* Corner weights L[a] = (1/4pi) \int_T phi_a(y) n.(x - y)/|x - y|^3 dS_y of the
 * flat triangle T = (r0, r1, r2) with outward normal n = (r1-r0)x(r2-r0)/|.|,
 * phi_a the linear hat function equal to 1 at corner a.
 *
 * Derivation (restated, Lindholm 1984): n.(x - y) = -zeta with zeta = n.(r0 - x)
 * constant on T.  Writing phi_a(y) = s_{a+1}/(2A) m.(y - r_{a+1}) with
 * m = n x e_{a+1}/|e_{a+1}| the inward normal of the opposite edge and using
 * \int_T 1/R^3 = Omega/zeta and \int_T (y - x_p)/R^3 = sum_b (n x shat_b) P_b
 * (divergence theorem in the plane, P_b = \int_{edge b} dl/R):
 *   L_a = s_{a+1}/(8 pi A) [ eta_{a+1} Omega - zeta sum_b (shat_{a+1}.shat_b) P_b ],
 *   eta_b = (n x shat_b).(r_b - x),
 *   P_b = ln((R_b + R_{b+1} + s_b)/(R_b + R_{b+1} - s_b)).
 * Edge b runs from r_b to r_{b+1}.  When x lies in the plane of T
 * (|zeta| <= 1e-13 sqrt(A)) every term vanishes and L = 0. */
void o_lindholm(const double* x, const double* r0, const double* r1, const double* r2, double* L) {
    const double* r[3] = {r0, r1, r2};
    double e[3][3], sh[3][3], slen[3], rho[3][3], R[3];
    for (int b = 0; b < 3; ++b) {
        vsub(r[(b + 1) % 3], r[b], e[b]);
        slen[b] = vnorm(e[b]);
        for (int d = 0; d < 3; ++d) sh[b][d] = e[b][d] / slen[b];
        vsub(r[b], x, rho[b]);
        R[b] = vnorm(rho[b]);
    }
    double nn[3], e02[3];
    vsub(r2, r0, e02);
    vcross(e[0], e02, nn);
    double twoA = vnorm(nn);
    double A = 0.5 * twoA;
    double n[3] = {nn[0] / twoA, nn[1] / twoA, nn[2] / twoA};
    double zeta = vdot(n, rho[0]);
    if (fabs(zeta) <= 1e-13 * sqrt(A)) { L[0] = L[1] = L[2] = 0.0; return; }
    double Omega = o_solid_angle(x, r0, r1, r2);
    double P[3], eta[3];
    for (int b = 0; b < 3; ++b) {
        double Rs = R[b] + R[(b + 1) % 3];
        P[b] = log((Rs + slen[b]) / (Rs - slen[b]));
        double m[3];
        vcross(n, sh[b], m);
        eta[b] = vdot(m, rho[b]);
    }
    for (int a = 0; a < 3; ++a) {
        int o = (a + 1) % 3;               /* edge opposite corner a */
        double sum = 0.0;
        for (int b = 0; b < 3; ++b) sum += vdot(sh[o], sh[b]) * P[b];
        L[a] = slen[o] / (8.0 * O_PI * A) * (eta[o] * Omega - zeta * sum);
    }
}

/* Psi_i = sum over triangles not containing node i of Omega_T(xi_i). */
static double psi_one(int64_t i, const double* xyz, int64_t T, const int32_t* tri) {
    double s = 0.0;
    for (int64_t t = 0; t < T; ++t) {
        const int32_t* v = tri + 3 * t;
        if (v[0] == i || v[1] == i || v[2] == i) continue;
        s += o_solid_angle(xyz + 3 * i, xyz + 3 * v[0], xyz + 3 * v[1], xyz + 3 * v[2]);
    }
    return s;
}

void o_psi(int64_t N, const double* xyz, int64_t T, const int32_t* tri, double* psi) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) psi[i] = psi_one(i, xyz, T, tri);
}

/* Psi at the listed nodes only: psi[nodes[q]] for q < n (other entries untouched). */
void o_psi_nodes(const double* xyz, int64_t T, const int32_t* tri, int64_t n, const int64_t* nodes, double* psi) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n; ++q) psi[nodes[q]] = psi_one(nodes[q], xyz, T, tri);
}

/* One full row of M: row[j] = M_ij for all j (row has N entries, zeroed here). */
static void dense_row(int64_t i, int64_t N, const double* xyz, int64_t T, const int32_t* tri,
                      const double* psi, double* row) {
    memset(row, 0, sizeof(double) * (size_t)N);
    for (int64_t t = 0; t < T; ++t) {
        const int32_t* v = tri + 3 * t;
        if (v[0] == i || v[1] == i || v[2] == i) continue;
        double L[3];
        o_lindholm(xyz + 3 * i, xyz + 3 * v[0], xyz + 3 * v[1], xyz + 3 * v[2], L);
        row[v[0]] += L[0]; row[v[1]] += L[1]; row[v[2]] += L[2];
    }
    row[i] += psi[i] / (4.0 * O_PI) - 1.0;
}

/* Dense M (N x N row-major). */
void o_dense_matrix(int64_t N, const double* xyz, int64_t T, const int32_t* tri,
                    const double* psi, double* M) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) dense_row(i, N, xyz, T, tri, psi, M + (size_t)i * N);
}

/* Selected rows of M: out[q*N + j] = M_{rows[q], j}. */
void o_dense_rows(int64_t N, const double* xyz, int64_t T, const int32_t* tri, const double* psi,
                  int64_t nrows, const int64_t* rows, double* out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nrows; ++q) dense_row(rows[q], N, xyz, T, tri, psi, out + (size_t)q * N);
}

/* y = M x for r right-hand sides, x and y r x N row-major; rows of M built on the fly. */
void o_dense_matvec(int64_t N, const double* xyz, int64_t T, const int32_t* tri, const double* psi,
                    int32_t r, const double* x, double* y) {
#pragma omp parallel
    {
        double* row = (double*)malloc(sizeof(double) * (size_t)N);
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < N; ++i) {
            dense_row(i, N, xyz, T, tri, psi, row);
            for (int32_t c = 0; c < r; ++c) {
                double s = 0.0;
                for (int64_t j = 0; j < N; ++j) s += row[j] * x[(size_t)c * N + j];
                y[(size_t)c * N + i] = s;
            }
        }
        free(row);
    }
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0, 1] (Newton iteration on P_q)             */
/* ------------------------------------------------------------------ */
void o_gauss_legendre01(int q, double* x, double* w) {
    for (int k = 0; k < q; ++k) {
        double z = cos(O_PI * (k + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= q; ++l) {
                double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1; p1 = p2;
            }
            double pq = (q == 0) ? 1.0 : (q == 1 ? z : p1);
            double pq1 = (q == 1) ? 1.0 : p0;   /* P_{q-1} */
            dp = q * (z * pq - pq1) / (z * z - 1.0);
            double dz = pq / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[k] = 0.5 * (1.0 - z);
        w[k] = 1.0 / ((1.0 - z * z) * dp * dp);   /* = 2/((1-z^2)P'^2) on [-1,1], halved */
    }
}

/* ------------------------------------------------------------------ */
/* Chebyshev interpolation on a box                                    */
/* ------------------------------------------------------------------ */

/* 1D Chebyshev points of the first kind on [lo, hi]: c + (w/2) cos((2k+1) pi/(2m)). */
static void cheb1d(double lo, double hi, int m, double* p) {
    double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
    for (int k = 0; k < m; ++k) p[k] = c + h * cos((2.0 * k + 1.0) * O_PI / (2.0 * m));
}

/* Lagrange polynomial l_k(t) for nodes p[0..m-1] and its derivative. */
static double lag(const double* p, int m, int k, double t) {
    double v = 1.0;
    for (int l = 0; l < m; ++l) if (l != k) v *= (t - p[l]) / (p[k] - p[l]);
    return v;
}
static double dlag(const double* p, int m, int k, double t) {
    double s = 0.0;
    for (int q = 0; q < m; ++q) {
        if (q == k) continue;
        double v = 1.0 / (p[k] - p[q]);
        for (int l = 0; l < m; ++l) if (l != k && l != q) v *= (t - p[l]) / (p[k] - p[l]);
        s += v;
    }
    return s;
}

/* Tensor Chebyshev points of a box (lo[3], hi[3]) -> pts[k*3], index
 * nu = (a*m + b)*m + c for axis points (a, b, c) (x slowest). */
void o_cheb_points(const double* box, int m, double* pts) {
    double px[16], py[16], pz[16];
    cheb1d(box[0], box[3], m, px); cheb1d(box[1], box[4], m, py); cheb1d(box[2], box[5], m, pz);
    for (int a = 0; a < m; ++a) for (int b = 0; b < m; ++b) for (int c = 0; c < m; ++c) {
        int nu = (a * m + b) * m + c;
        pts[3 * nu] = px[a]; pts[3 * nu + 1] = py[b]; pts[3 * nu + 2] = pz[c];
    }
}

/* L_nu(x) for all nu (out[k]) and optionally grad L_nu(x) (grad[3k]). */
void o_lagrange3(const double* box, int m, const double* x, double* out, double* grad) {
    double px[16], py[16], pz[16];
    cheb1d(box[0], box[3], m, px); cheb1d(box[1], box[4], m, py); cheb1d(box[2], box[5], m, pz);
    double lx[16], ly[16], lz[16], dx[16], dy[16], dz[16];
    for (int a = 0; a < m; ++a) {
        lx[a] = lag(px, m, a, x[0]); ly[a] = lag(py, m, a, x[1]); lz[a] = lag(pz, m, a, x[2]);
        dx[a] = dlag(px, m, a, x[0]); dy[a] = dlag(py, m, a, x[1]); dz[a] = dlag(pz, m, a, x[2]);
    }
    for (int a = 0; a < m; ++a) for (int b = 0; b < m; ++b) for (int c = 0; c < m; ++c) {
        int nu = (a * m + b) * m + c;
        if (out) out[nu] = lx[a] * ly[b] * lz[c];
        if (grad) {
            grad[3 * nu] = dx[a] * ly[b] * lz[c];
            grad[3 * nu + 1] = lx[a] * dy[b] * lz[c];
            grad[3 * nu + 2] = lx[a] * ly[b] * dz[c];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Oracle H2 object                                                    */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t N, T;
    double* xyz;
    int32_t* tri;
    double* psi;
    /* node -> triangle adjacency (CSR) */
    int64_t* adj_ptr;
    int32_t* adj;
    /* parameters */
    int m, k, leaf, q;
    double eta, rho;
    /* cluster tree, numbered level by level (root = 0) */
    int nc, nlevels;
    int32_t *perm, *start, *size, *parent, *child0, *child1, *level;
    double* box;      /* 6 per cluster: lo[3], hi[3] (inflated support box) */
    /* block partition */
    int64_t nfar, nnear;
    int32_t *far_t, *far_s, *near_t, *near_s;
    /* stored data (store != 0) */
    int store;
    double** near_val;   /* per near block |t| x |s| row-major, includes D on the diagonal */
    double** Vd;         /* per cluster |t| x k (NULL when unused) */
    double** Wd;         /* per cluster |s| x k (NULL when unused) */
    char *is_tgt, *is_src;
} o2_t;

static void build_adjacency(o2_t* o) {
    o->adj_ptr = (int64_t*)calloc((size_t)o->N + 1, sizeof(int64_t));
    for (int64_t t = 0; t < o->T; ++t)
        for (int a = 0; a < 3; ++a) o->adj_ptr[o->tri[3 * t + a] + 1]++;
    for (int64_t i = 0; i < o->N; ++i) o->adj_ptr[i + 1] += o->adj_ptr[i];
    o->adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)o->adj_ptr[o->N]);
    int64_t* fill = (int64_t*)calloc((size_t)o->N, sizeof(int64_t));
    for (int64_t t = 0; t < o->T; ++t)
        for (int a = 0; a < 3; ++a) {
            int32_t v = o->tri[3 * t + a];
            o->adj[o->adj_ptr[v] + fill[v]++] = (int32_t)t;
        }
    free(fill);
}

/* Cluster tree: bisect the bounding box of a cluster's nodes at the midpoint
 * (lo+hi)/2 of its longest side (lowest axis on ties); nodes with coordinate
 * <= mid go to the first child, keeping their order; stop at size <= leaf.
 * Each cluster's box is the bounding box of all triangles adjacent to its
 * nodes, each side widened about its centre to at least rho * longest side. */
static void build_tree(o2_t* o) {
    int64_t N = o->N;
    int cap = (int)(2 * N + 1);
    o->perm = (int32_t*)malloc(sizeof(int32_t) * N);
    o->start = (int32_t*)malloc(sizeof(int32_t) * cap);
    o->size = (int32_t*)malloc(sizeof(int32_t) * cap);
    o->parent = (int32_t*)malloc(sizeof(int32_t) * cap);
    o->child0 = (int32_t*)malloc(sizeof(int32_t) * cap);
    o->child1 = (int32_t*)malloc(sizeof(int32_t) * cap);
    o->level = (int32_t*)malloc(sizeof(int32_t) * cap);
    o->box = (double*)malloc(sizeof(double) * 6 * cap);
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * N);
    for (int64_t i = 0; i < N; ++i) o->perm[i] = (int32_t)i;
    int nc = 1;
    o->start[0] = 0; o->size[0] = (int32_t)N; o->parent[0] = -1; o->level[0] = 0;
    for (int c = 0; c < nc; ++c) {   /* queue order = level order */
        int32_t st = o->start[c], sz = o->size[c];
        o->child0[c] = o->child1[c] = -1;
        /* support box */
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int32_t q = st; q < st + sz; ++q) {
            int32_t i = o->perm[q];
            for (int64_t p = o->adj_ptr[i]; p < o->adj_ptr[i + 1]; ++p) {
                const int32_t* v = o->tri + 3 * (int64_t)o->adj[p];
                for (int a = 0; a < 3; ++a)
                    for (int d = 0; d < 3; ++d) {
                        double z = o->xyz[3 * (int64_t)v[a] + d];
                        if (z < lo[d]) lo[d] = z;
                        if (z > hi[d]) hi[d] = z;
                    }
            }
        }
        double longest = 0.0;
        for (int d = 0; d < 3; ++d) if (hi[d] - lo[d] > longest) longest = hi[d] - lo[d];
        for (int d = 0; d < 3; ++d) {
            double minw = o->rho * longest;
            if (hi[d] - lo[d] < minw) {
                double cen = 0.5 * (lo[d] + hi[d]);
                lo[d] = cen - 0.5 * minw;
                hi[d] = cen + 0.5 * minw;
            }
            o->box[6 * c + d] = lo[d];
            o->box[6 * c + 3 + d] = hi[d];
        }
        if (sz <= o->leaf) continue;
        /* split on the node bounding box */
        double nlo[3] = {INFINITY, INFINITY, INFINITY}, nhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int32_t q = st; q < st + sz; ++q)
            for (int d = 0; d < 3; ++d) {
                double z = o->xyz[3 * (int64_t)o->perm[q] + d];
                if (z < nlo[d]) nlo[d] = z;
                if (z > nhi[d]) nhi[d] = z;
            }
        int ax = 0;
        for (int d = 1; d < 3; ++d) if (nhi[d] - nlo[d] > nhi[ax] - nlo[ax]) ax = d;
        double mid = (nlo[ax] + nhi[ax]) / 2.0;
        int32_t n0 = 0, n1 = 0;
        for (int32_t q = st; q < st + sz; ++q)
            if (o->xyz[3 * (int64_t)o->perm[q] + ax] <= mid) n0++;
        if (n0 == 0 || n0 == sz) continue;   /* coincident nodes: keep as leaf */
        for (int32_t q = st; q < st + sz; ++q) {
            int32_t i = o->perm[q];
            if (o->xyz[3 * (int64_t)i + ax] <= mid) tmp[n1++] = i;
        }
        for (int32_t q = st; q < st + sz; ++q) {
            int32_t i = o->perm[q];
            if (!(o->xyz[3 * (int64_t)i + ax] <= mid)) tmp[n1++] = i;
        }
        memcpy(o->perm + st, tmp, sizeof(int32_t) * sz);
        for (int h = 0; h < 2; ++h) {
            int ch = nc++;
            o->start[ch] = h == 0 ? st : st + n0;
            o->size[ch] = h == 0 ? n0 : sz - n0;
            o->parent[ch] = c;
            o->level[ch] = o->level[c] + 1;
            if (h == 0) o->child0[c] = ch; else o->child1[c] = ch;
        }
    }
    o->nc = nc;
    int L = 0;
    for (int c = 0; c < nc; ++c) if (o->level[c] > L) L = o->level[c];
    o->nlevels = L + 1;
    free(tmp);
}

static double box_diam(const double* b) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) s += (b[3 + d] - b[d]) * (b[3 + d] - b[d]);
    return sqrt(s);
}
static double box_dist(const double* a, const double* b) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double g = 0.0;
        if (b[d] > a[3 + d]) g = b[d] - a[3 + d];
        else if (a[d] > b[3 + d]) g = a[d] - b[3 + d];
        s += g * g;
    }
    return sqrt(s);
}
int o_admissible(const double* bt, const double* bs, double eta) {
    double dt = box_diam(bt), ds = box_diam(bs);
    double dm = dt > ds ? dt : ds;
    return dm <= eta * box_dist(bt, bs);
}

/* Block partition by recursion from (root, root): admissible -> far; both
 * leaves -> near; otherwise recurse into children(t) x children(s), where a
 * leaf stands for itself. */
static void build_blocks(o2_t* o) {
    int64_t cap_far = 1024, cap_near = 1024, cap_st = 1024;
    o->far_t = (int32_t*)malloc(sizeof(int32_t) * cap_far);
    o->far_s = (int32_t*)malloc(sizeof(int32_t) * cap_far);
    o->near_t = (int32_t*)malloc(sizeof(int32_t) * cap_near);
    o->near_s = (int32_t*)malloc(sizeof(int32_t) * cap_near);
    int32_t* st = (int32_t*)malloc(sizeof(int32_t) * 2 * cap_st);
    int64_t sp = 0, nf = 0, nn = 0;
    st[0] = 0; st[1] = 0; sp = 1;
    while (sp > 0) {
        --sp;
        int32_t t = st[2 * sp], s = st[2 * sp + 1];
        int leaf_t = o->child0[t] < 0, leaf_s = o->child0[s] < 0;
        if (o_admissible(o->box + 6 * t, o->box + 6 * s, o->eta)) {
            if (nf == cap_far) {
                cap_far *= 2;
                o->far_t = (int32_t*)realloc(o->far_t, sizeof(int32_t) * cap_far);
                o->far_s = (int32_t*)realloc(o->far_s, sizeof(int32_t) * cap_far);
            }
            o->far_t[nf] = t; o->far_s[nf] = s; nf++;
        } else if (leaf_t && leaf_s) {
            if (nn == cap_near) {
                cap_near *= 2;
                o->near_t = (int32_t*)realloc(o->near_t, sizeof(int32_t) * cap_near);
                o->near_s = (int32_t*)realloc(o->near_s, sizeof(int32_t) * cap_near);
            }
            o->near_t[nn] = t; o->near_s[nn] = s; nn++;
        } else {
            int32_t ct[2], cs[2];
            int nt = 0, ns = 0;
            if (leaf_t) ct[nt++] = t; else { ct[nt++] = o->child0[t]; ct[nt++] = o->child1[t]; }
            if (leaf_s) cs[ns++] = s; else { cs[ns++] = o->child0[s]; cs[ns++] = o->child1[s]; }
            /* push in reverse so that (first child, first child) is processed first */
            for (int a = nt - 1; a >= 0; --a)
                for (int b = ns - 1; b >= 0; --b) {
                    if (sp == cap_st) { cap_st *= 2; st = (int32_t*)realloc(st, sizeof(int32_t) * 2 * cap_st); }
                    st[2 * sp] = ct[a]; st[2 * sp + 1] = cs[b]; sp++;
                }
        }
    }
    free(st);
    o->nfar = nf; o->nnear = nn;
}

/* V_t(i, nu) = L^t_nu(xi_i) for the nodes of cluster t, |t| x k row-major. */
static double* make_V(const o2_t* o, int c) {
    int32_t sz = o->size[c];
    double* V = (double*)malloc(sizeof(double) * (size_t)sz * o->k);
    for (int32_t q = 0; q < sz; ++q) {
        int32_t i = o->perm[o->start[c] + q];
        o_lagrange3(o->box + 6 * c, o->m, o->xyz + 3 * (int64_t)i, V + (size_t)q * o->k, NULL);
    }
    return V;
}

/* W_s(j, mu) = sum_{T containing j} \int_T phi_j n_T . grad L^s_mu dS, for the
 * nodes of cluster s, |s| x k row-major.  Collapsed (Duffy) Gauss-Legendre
 * product rule with q points per direction on each triangle. */
static void w_row(const o2_t* o, const double* box, int32_t j, int q, const double* gx,
                  const double* gw, double* row) {
    int k = o->k;
    double* grad = (double*)malloc(sizeof(double) * 3 * k);
    for (int mu = 0; mu < k; ++mu) row[mu] = 0.0;
    for (int64_t p = o->adj_ptr[j]; p < o->adj_ptr[j + 1]; ++p) {
        const int32_t* v = o->tri + 3 * (int64_t)o->adj[p];
        int cj = v[0] == j ? 0 : (v[1] == j ? 1 : 2);
        const double *a = o->xyz + 3 * (int64_t)v[0], *b = o->xyz + 3 * (int64_t)v[1],
                     *c = o->xyz + 3 * (int64_t)v[2];
        double e1[3], e2[3], nn[3];
        vsub(b, a, e1); vsub(c, a, e2); vcross(e1, e2, nn);
        double twoA = vnorm(nn);
        double n[3] = {nn[0] / twoA, nn[1] / twoA, nn[2] / twoA};
        for (int iu = 0; iu < q; ++iu)
            for (int iv = 0; iv < q; ++iv) {
                double s = gx[iu], t = gx[iv] * (1.0 - gx[iu]);
                double wt = gw[iu] * gw[iv] * (1.0 - gx[iu]) * twoA;
                double phi[3] = {1.0 - s - t, s, t};
                double y[3];
                for (int d = 0; d < 3; ++d) y[d] = a[d] + s * e1[d] + t * e2[d];
                o_lagrange3(box, o->m, y, NULL, grad);
                for (int mu = 0; mu < k; ++mu)
                    row[mu] += wt * phi[cj] * vdot(n, grad + 3 * mu);
            }
    }
    free(grad);
}

static double* make_W(const o2_t* o, int c) {
    int32_t sz = o->size[c];
    double* W = (double*)malloc(sizeof(double) * (size_t)sz * o->k);
    double gx[64], gw[64];
    o_gauss_legendre01(o->q, gx, gw);
    for (int32_t q = 0; q < sz; ++q)
        w_row(o, o->box + 6 * c, o->perm[o->start[c] + q], o->q, gx, gw, W + (size_t)q * o->k);
    return W;
}

/* K_ij + D_ij for one pair (i, j) by summing the corner weights of the
 * triangles around j that do not contain i. */
static double entry(const o2_t* o, int32_t i, int32_t j) {
    double s = 0.0;
    for (int64_t p = o->adj_ptr[j]; p < o->adj_ptr[j + 1]; ++p) {
        const int32_t* v = o->tri + 3 * (int64_t)o->adj[p];
        if (v[0] == i || v[1] == i || v[2] == i) continue;
        double L[3];
        o_lindholm(o->xyz + 3 * (int64_t)i, o->xyz + 3 * (int64_t)v[0], o->xyz + 3 * (int64_t)v[1],
                   o->xyz + 3 * (int64_t)v[2], L);
        s += v[0] == j ? L[0] : (v[1] == j ? L[1] : L[2]);
    }
    if (i == j) s += o->psi[i] / (4.0 * O_PI) - 1.0;
    return s;
}

void o2_destroy(void* h);

void* o2_create(int64_t N, const double* xyz, int64_t T, const int32_t* tri, int32_t m,
                int32_t leaf, double eta, double rho, int32_t q, int32_t store) {
    o2_t* o = (o2_t*)calloc(1, sizeof(o2_t));
    o->N = N; o->T = T;
    o->xyz = (double*)malloc(sizeof(double) * 3 * N);
    memcpy(o->xyz, xyz, sizeof(double) * 3 * N);
    o->tri = (int32_t*)malloc(sizeof(int32_t) * 3 * T);
    memcpy(o->tri, tri, sizeof(int32_t) * 3 * T);
    o->m = m; o->k = m * m * m; o->leaf = leaf; o->eta = eta; o->rho = rho;
    o->q = q > 0 ? q : (3 * m - 1 + 1) / 2;   /* ceil((3m-1)/2) */
    o->psi = (double*)malloc(sizeof(double) * N);
    if (store) {
        o_psi(N, o->xyz, T, o->tri, o->psi);
    } else {   /* sampled rows: Psi is evaluated for the sampled nodes only (o2_rows) */
        for (int64_t i = 0; i < N; ++i) o->psi[i] = NAN;
    }
    build_adjacency(o);
    build_tree(o);
    build_blocks(o);
    o->is_tgt = (char*)calloc(o->nc, 1);
    o->is_src = (char*)calloc(o->nc, 1);
    for (int64_t b = 0; b < o->nfar; ++b) { o->is_tgt[o->far_t[b]] = 1; o->is_src[o->far_s[b]] = 1; }
    o->Vd = (double**)calloc(o->nc, sizeof(double*));
    o->Wd = (double**)calloc(o->nc, sizeof(double*));
    o->store = store;
    if (store) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < o->nc; ++c) {
            if (o->is_tgt[c]) o->Vd[c] = make_V(o, c);
            if (o->is_src[c]) o->Wd[c] = make_W(o, c);
        }
        o->near_val = (double**)calloc(o->nnear, sizeof(double*));
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t b = 0; b < o->nnear; ++b) {
            int32_t t = o->near_t[b], s = o->near_s[b];
            double* B = (double*)malloc(sizeof(double) * (size_t)o->size[t] * o->size[s]);
            for (int32_t a = 0; a < o->size[t]; ++a)
                for (int32_t c = 0; c < o->size[s]; ++c)
                    B[(size_t)a * o->size[s] + c] =
                        entry(o, o->perm[o->start[t] + a], o->perm[o->start[s] + c]);
            o->near_val[b] = B;
        }
    }
    return o;
}

/* info[0..7] = nc, nlevels, nfar, nnear, near entries, far coefficient count (nfar k^2), k, q */
void o2_info(void* h, int64_t* info) {
    o2_t* o = (o2_t*)h;
    int64_t ne = 0;
    for (int64_t b = 0; b < o->nnear; ++b) ne += (int64_t)o->size[o->near_t[b]] * o->size[o->near_s[b]];
    info[0] = o->nc; info[1] = o->nlevels; info[2] = o->nfar; info[3] = o->nnear;
    info[4] = ne; info[5] = o->nfar * (int64_t)o->k * o->k; info[6] = o->k; info[7] = o->q;
}

void o2_get_tree(void* h, int32_t* perm, int32_t* start, int32_t* size, int32_t* parent,
                 int32_t* child0, int32_t* child1, int32_t* level, double* box) {
    o2_t* o = (o2_t*)h;
    memcpy(perm, o->perm, sizeof(int32_t) * o->N);
    memcpy(start, o->start, sizeof(int32_t) * o->nc);
    memcpy(size, o->size, sizeof(int32_t) * o->nc);
    memcpy(parent, o->parent, sizeof(int32_t) * o->nc);
    memcpy(child0, o->child0, sizeof(int32_t) * o->nc);
    memcpy(child1, o->child1, sizeof(int32_t) * o->nc);
    memcpy(level, o->level, sizeof(int32_t) * o->nc);
    memcpy(box, o->box, sizeof(double) * 6 * o->nc);
}

void o2_get_blocks(void* h, int32_t* far_t, int32_t* far_s, int32_t* near_t, int32_t* near_s) {
    o2_t* o = (o2_t*)h;
    memcpy(far_t, o->far_t, sizeof(int32_t) * o->nfar);
    memcpy(far_s, o->far_s, sizeof(int32_t) * o->nfar);
    memcpy(near_t, o->near_t, sizeof(int32_t) * o->nnear);
    memcpy(near_s, o->near_s, sizeof(int32_t) * o->nnear);
}

void o2_get_psi(void* h, double* psi) {
    o2_t* o = (o2_t*)h;
    memcpy(psi, o->psi, sizeof(double) * o->N);
}

/* Direct bases of one cluster (|c| x k row-major each); either output may be NULL. */
void o2_cluster_bases(void* h, int32_t c, double* V, double* W) {
    o2_t* o = (o2_t*)h;
    if (V) { double* t = make_V(o, c); memcpy(V, t, sizeof(double) * o->size[c] * o->k); free(t); }
    if (W) { double* t = make_W(o, c); memcpy(W, t, sizeof(double) * o->size[c] * o->k); free(t); }
}

/* S_ts (k x k row-major): g(x^t_nu, x^s_mu) = 1/(4 pi |x^t_nu - x^s_mu|). */
static void make_S(const o2_t* o, int32_t t, int32_t s, double* S) {
    int k = o->k;
    double* pt = (double*)malloc(sizeof(double) * 3 * k);
    double* ps = (double*)malloc(sizeof(double) * 3 * k);
    o_cheb_points(o->box + 6 * t, o->m, pt);
    o_cheb_points(o->box + 6 * s, o->m, ps);
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            double d[3];
            vsub(pt + 3 * a, ps + 3 * b, d);
            S[a * k + b] = 1.0 / (4.0 * O_PI * vnorm(d));
        }
    free(pt); free(ps);
}

void o2_coupling(void* h, int32_t t, int32_t s, double* S) { make_S((o2_t*)h, t, s, S); }

/* y = (near part + far part) x for r right-hand sides (r x N row-major).
 * Far part: for every admissible block, y|_t += V_t (S_ts (W_s^T x|_s)). */
void o2_matvec(void* h, int32_t r, const double* x, double* y) {
    o2_t* o = (o2_t*)h;
    int64_t N = o->N;
    int k = o->k;
    memset(y, 0, sizeof(double) * (size_t)r * N);
    /* near blocks, grouped by target so that the row updates do not race */
    int64_t* cnt = (int64_t*)calloc(o->nc + 1, sizeof(int64_t));
    for (int64_t b = 0; b < o->nnear; ++b) cnt[o->near_t[b] + 1]++;
    for (int c = 0; c < o->nc; ++c) cnt[c + 1] += cnt[c];
    int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (o->nnear + 1));
    int64_t* fill = (int64_t*)calloc((size_t)o->nc + 1, sizeof(int64_t));
    for (int64_t b = 0; b < o->nnear; ++b) ord[cnt[o->near_t[b]] + fill[o->near_t[b]]++] = b;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < o->nc; ++c) {
        for (int64_t p = cnt[c]; p < cnt[c + 1]; ++p) {
            int64_t b = ord[p];
            int32_t t = o->near_t[b], s = o->near_s[b];
            const double* B = o->near_val[b];
            for (int32_t cc = 0; cc < r; ++cc)
                for (int32_t a = 0; a < o->size[t]; ++a) {
                    double acc = 0.0;
                    for (int32_t j = 0; j < o->size[s]; ++j)
                        acc += B[(size_t)a * o->size[s] + j] *
                               x[(size_t)cc * N + o->perm[o->start[s] + j]];
                    y[(size_t)cc * N + o->perm[o->start[t] + a]] += acc;
                }
        }
    }
    free(cnt); free(ord); free(fill);
    /* far blocks: xhat_s = W_s^T x|_s per source cluster */
    double** xh = (double**)calloc(o->nc, sizeof(double*));
    double** yh = (double**)calloc(o->nc, sizeof(double*));
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < o->nc; ++c) {
        if (o->is_src[c]) {
            double* v = (double*)calloc((size_t)k * r, sizeof(double));
            for (int32_t cc = 0; cc < r; ++cc)
                for (int32_t j = 0; j < o->size[c]; ++j) {
                    double xj = x[(size_t)cc * N + o->perm[o->start[c] + j]];
                    for (int mu = 0; mu < k; ++mu) v[cc * k + mu] += o->Wd[c][(size_t)j * k + mu] * xj;
                }
            xh[c] = v;
        }
        if (o->is_tgt[c]) yh[c] = (double*)calloc((size_t)k * r, sizeof(double));
    }
    /* yhat_t += S_ts xhat_s, grouped by target */
    int64_t* fc = (int64_t*)calloc(o->nc + 1, sizeof(int64_t));
    for (int64_t b = 0; b < o->nfar; ++b) fc[o->far_t[b] + 1]++;
    for (int c = 0; c < o->nc; ++c) fc[c + 1] += fc[c];
    int64_t* ford = (int64_t*)malloc(sizeof(int64_t) * (o->nfar + 1));
    int64_t* ff = (int64_t*)calloc((size_t)o->nc + 1, sizeof(int64_t));
    for (int64_t b = 0; b < o->nfar; ++b) ford[fc[o->far_t[b]] + ff[o->far_t[b]]++] = b;
#pragma omp parallel
    {
        double* S = (double*)malloc(sizeof(double) * k * k);
#pragma omp for schedule(dynamic, 1)
        for (int c = 0; c < o->nc; ++c) {
            for (int64_t p = fc[c]; p < fc[c + 1]; ++p) {
                int64_t b = ford[p];
                int32_t s = o->far_s[b];
                make_S(o, c, s, S);
                for (int32_t cc = 0; cc < r; ++cc)
                    for (int a = 0; a < k; ++a) {
                        double acc = 0.0;
                        for (int bb = 0; bb < k; ++bb) acc += S[a * k + bb] * xh[s][cc * k + bb];
                        yh[c][cc * k + a] += acc;
                    }
            }
        }
        free(S);
    }
    free(fc); free(ford); free(ff);
    /* y|_t += V_t yhat_t; clusters of one level are disjoint, so loop levels */
    for (int lv = 0; lv < o->nlevels; ++lv) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < o->nc; ++c) {
            if (o->level[c] != lv || !o->is_tgt[c]) continue;
            for (int32_t cc = 0; cc < r; ++cc)
                for (int32_t a = 0; a < o->size[c]; ++a) {
                    double acc = 0.0;
                    for (int nu = 0; nu < k; ++nu) acc += o->Vd[c][(size_t)a * k + nu] * yh[c][cc * k + nu];
                    y[(size_t)cc * N + o->perm[o->start[c] + a]] += acc;
                }
        }
    }
    for (int c = 0; c < o->nc; ++c) { free(xh[c]); free(yh[c]); }
    free(xh); free(yh);
}

/* Selected rows of the H2 approximation applied to x (works with store == 0):
 * out[cc*nrows + q] = (H2 x)_{rows[q]} for right-hand side cc.  Near entries
 * and bases are evaluated on the fly. */
void o2_rows(void* h, int32_t r, const double* x, int64_t nrows, const int64_t* rows, double* out) {
    o2_t* o = (o2_t*)h;
    int64_t N = o->N;
    int k = o->k;
    int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * N);      /* node -> position in perm */
    for (int64_t q = 0; q < N; ++q) pos[o->perm[q]] = (int32_t)q;
    int32_t* leaf_of = (int32_t*)malloc(sizeof(int32_t) * N);  /* position -> leaf cluster */
    for (int c = 0; c < o->nc; ++c)
        if (o->child0[c] < 0)
            for (int32_t q = o->start[c]; q < o->start[c] + o->size[c]; ++q) leaf_of[q] = c;
    /* sources needed by the sampled rows */
    char* need = (char*)calloc(o->nc, 1);
    char* on_path = (char*)calloc(o->nc, 1);
    for (int64_t q = 0; q < nrows; ++q) {
        for (int c = leaf_of[pos[rows[q]]]; c >= 0; c = o->parent[c]) on_path[c] = 1;
    }
    for (int64_t b = 0; b < o->nfar; ++b) if (on_path[o->far_t[b]]) need[o->far_s[b]] = 1;
    /* Psi at the sampled nodes (all nodes already have it when the near field is stored) */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nrows; ++q)
        if (isnan(o->psi[rows[q]])) o->psi[rows[q]] = psi_one(rows[q], o->xyz, o->T, o->tri);
    double** xh = (double**)calloc(o->nc, sizeof(double*));
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < o->nc; ++c) {
        if (!need[c]) continue;
        double* W = make_W(o, c);
        double* v = (double*)calloc((size_t)k * r, sizeof(double));
        for (int32_t cc = 0; cc < r; ++cc)
            for (int32_t j = 0; j < o->size[c]; ++j) {
                double xj = x[(size_t)cc * N + o->perm[o->start[c] + j]];
                for (int mu = 0; mu < k; ++mu) v[cc * k + mu] += W[(size_t)j * k + mu] * xj;
            }
        free(W);
        xh[c] = v;
    }
#pragma omp parallel
    {
        double* S = (double*)malloc(sizeof(double) * k * k);
        double* Lv = (double*)malloc(sizeof(double) * k);
        double* tmp = (double*)malloc(sizeof(double) * k);
#pragma omp for schedule(dynamic, 1)
        for (int64_t q = 0; q < nrows; ++q) {
            int32_t i = (int32_t)rows[q];
            for (int32_t cc = 0; cc < r; ++cc) out[(size_t)cc * nrows + q] = 0.0;
            int32_t lt = leaf_of[pos[i]];
            /* near blocks of the leaf containing i */
            for (int64_t b = 0; b < o->nnear; ++b) {
                if (o->near_t[b] != lt) continue;
                int32_t s = o->near_s[b];
                for (int32_t j = 0; j < o->size[s]; ++j) {
                    int32_t jj = o->perm[o->start[s] + j];
                    double e = entry(o, i, jj);
                    for (int32_t cc = 0; cc < r; ++cc) out[(size_t)cc * nrows + q] += e * x[(size_t)cc * N + jj];
                }
            }
            /* far blocks whose target contains i */
            for (int64_t b = 0; b < o->nfar; ++b) {
                int32_t t = o->far_t[b], s = o->far_s[b];
                int32_t p = pos[i];
                if (p < o->start[t] || p >= o->start[t] + o->size[t]) continue;
                make_S(o, t, s, S);
                o_lagrange3(o->box + 6 * t, o->m, o->xyz + 3 * (int64_t)i, Lv, NULL);
                for (int32_t cc = 0; cc < r; ++cc) {
                    for (int a = 0; a < k; ++a) {
                        double acc = 0.0;
                        for (int bb = 0; bb < k; ++bb) acc += S[a * k + bb] * xh[s][cc * k + bb];
                        tmp[a] = acc;
                    }
                    double acc = 0.0;
                    for (int a = 0; a < k; ++a) acc += Lv[a] * tmp[a];
                    out[(size_t)cc * nrows + q] += acc;
                }
            }
        }
        free(S); free(Lv); free(tmp);
    }
    for (int c = 0; c < o->nc; ++c) free(xh[c]);
    free(xh); free(need); free(on_path); free(pos); free(leaf_of);
}

void o2_destroy(void* h) {
    o2_t* o = (o2_t*)h;
    if (!o) return;
    if (o->near_val) { for (int64_t b = 0; b < o->nnear; ++b) free(o->near_val[b]); free(o->near_val); }
    if (o->Vd) { for (int c = 0; c < o->nc; ++c) free(o->Vd[c]); free(o->Vd); }
    if (o->Wd) { for (int c = 0; c < o->nc; ++c) free(o->Wd[c]); free(o->Wd); }
    free(o->is_tgt); free(o->is_src);
    free(o->far_t); free(o->far_s); free(o->near_t); free(o->near_s);
    free(o->perm); free(o->start); free(o->size); free(o->parent); free(o->child0); free(o->child1);
    free(o->level); free(o->box);
    free(o->adj_ptr); free(o->adj);
    free(o->xyz); free(o->tri); free(o->psi);
    free(o);
}
