// Host-side construction of the H2 structure: mesh validation, geometric
// cluster tree and eta-admissible block partition (arXiv:1811.05731, Section
// "H2-Matrix Compression": a block K|t x s is compressed when its two
// clusters are geometrically well separated and kept exactly otherwise).  These are index and
// comparison computations done once per operator; all numeric assembly and
// the matrix-vector product run in CUDA kernels.
//
// This file is compiled with -ffp-contract=off so that box widths, diameters
// and distances are rounded the same way on every host architecture: the
// tree and the block partition are deterministic functions of the mesh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <utility>

#include "h2_internal.h"

namespace h2 {

namespace {

inline double tri_cross_norm(const double* a, const double* b, const double* c, double* n) {
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    n[0] = u[1] * v[2] - u[2] * v[1];
    n[1] = u[2] * v[0] - u[0] * v[2];
    n[2] = u[0] * v[1] - u[1] * v[0];
    return std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
}

}  // namespace

// Checks that the mesh is a closed, consistently outward-oriented surface
// without degenerate triangles, and builds the node -> triangle adjacency.
int validate_mesh(const double* xyz, int64_t N, const int32_t* tri, int64_t T,
                  std::vector<int64_t>& adj_ptr, std::vector<int32_t>& adj) {
    if (N < 4 || T < 4) return H2_ERR_INVALID_ARG;
    if (N > (int64_t)1 << 30 || T > (int64_t)1 << 30) return H2_ERR_INVALID_ARG;
    for (int64_t t = 0; t < T; ++t) {
        const int32_t* v = tri + 3 * t;
        for (int a = 0; a < 3; ++a)
            if (v[a] < 0 || v[a] >= N) return H2_ERR_INVALID_ARG;
        if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return H2_ERR_DEGENERATE_TRIANGLE;
        double n[3];
        const double *p0 = xyz + 3 * (int64_t)v[0], *p1 = xyz + 3 * (int64_t)v[1],
                     *p2 = xyz + 3 * (int64_t)v[2];
        double len2 = 0.0;   // longest edge, squared
        const double* P[3] = {p0, p1, p2};
        for (int a = 0; a < 3; ++a) {
            double e2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double e = P[(a + 1) % 3][d] - P[a][d];
                e2 += e * e;
            }
            len2 = std::max(len2, e2);
        }
        double twoA = tri_cross_norm(p0, p1, p2, n);
        if (!(twoA > 1e-12 * len2)) return H2_ERR_DEGENERATE_TRIANGLE;
    }
    // every directed edge a->b must appear once and its reverse b->a once
    std::vector<std::pair<int64_t, int64_t>> edges;
    edges.reserve((size_t)(3 * T));
    for (int64_t t = 0; t < T; ++t)
        for (int a = 0; a < 3; ++a) edges.emplace_back(tri[3 * t + a], tri[3 * t + (a + 1) % 3]);
    std::vector<std::pair<int64_t, int64_t>> sorted = edges;
    std::sort(sorted.begin(), sorted.end());
    for (size_t i = 1; i < sorted.size(); ++i)
        if (sorted[i] == sorted[i - 1]) return H2_ERR_MESH_ORIENTATION;
    for (const auto& e : edges) {
        std::pair<int64_t, int64_t> rev(e.second, e.first);
        if (!std::binary_search(sorted.begin(), sorted.end(), rev)) {
            // the undirected edge exists twice with the same direction -> orientation,
            // otherwise the surface is open
            return H2_ERR_MESH_OPEN;
        }
    }
    // enclosed volume must be positive (outward normals)
    double vol = 0.0;
    for (int64_t t = 0; t < T; ++t) {
        const double *a = xyz + 3 * (int64_t)tri[3 * t], *b = xyz + 3 * (int64_t)tri[3 * t + 1],
                     *c = xyz + 3 * (int64_t)tri[3 * t + 2];
        vol += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
               a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    if (!(vol > 0.0)) return H2_ERR_MESH_ORIENTATION;
    adj_ptr.assign((size_t)N + 1, 0);
    for (int64_t t = 0; t < T; ++t)
        for (int a = 0; a < 3; ++a) adj_ptr[tri[3 * t + a] + 1]++;
    for (int64_t i = 0; i < N; ++i) {
        if (adj_ptr[i + 1] == 0) return H2_ERR_MESH_OPEN;   // unreferenced node
        adj_ptr[i + 1] += adj_ptr[i];
    }
    adj.assign((size_t)adj_ptr[N], 0);
    std::vector<int64_t> fill(adj_ptr.begin(), adj_ptr.end() - 1);
    for (int64_t t = 0; t < T; ++t)
        for (int a = 0; a < 3; ++a) adj[fill[tri[3 * t + a]]++] = (int32_t)t;
    // the triangles around every node must form one fan: the link edges
    // (a -> b for a triangle (i, a, b)) close into a single cycle.  The solid
    // angle at the node is computed from that cycle.
    std::vector<int32_t> ea, eb;
    for (int64_t i = 0; i < N; ++i) {
        ea.clear();
        eb.clear();
        for (int64_t p = adj_ptr[i]; p < adj_ptr[i + 1]; ++p) {
            const int32_t* v = tri + 3 * (int64_t)adj[p];
            const int c = v[0] == i ? 0 : (v[1] == i ? 1 : 2);
            ea.push_back(v[(c + 1) % 3]);
            eb.push_back(v[(c + 2) % 3]);
        }
        const size_t deg = ea.size();
        size_t cur = 0, steps = 0;
        do {
            size_t nxt = deg;
            for (size_t q = 0; q < deg; ++q)
                if (ea[q] == eb[cur]) { nxt = q; break; }
            if (nxt == deg) return H2_ERR_MESH_OPEN;
            cur = nxt;
            ++steps;
        } while (cur != 0 && steps <= deg);
        if (steps != deg) return H2_ERR_MESH_OPEN;
    }
    return H2_OK;
}

// Geometric cluster tree over the nodes, numbered level by level.
//  - split: the bounding box of the cluster's nodes is bisected at the
//    midpoint (lo + hi)/2 of its longest side (lowest axis index on ties);
//    nodes with coordinate <= midpoint form the first child, both children
//    keep the input order; clusters with at most `leaf` nodes are leaves.
//  - box: bounding box of all triangles touching the cluster's nodes (the
//    support of their basis functions), every side widened about its centre
//    to at least rho times the longest side so that the interpolation points
//    never collapse on flat faces.
void build_cluster_tree(h2_handle* op) {
    const h2_handle* g = op->geom;
    const int64_t N = g->N;
    const double* X = g->xyz.data();
    const double rho = op->params.box_inflation;
    const int leaf = op->params.leaf;

    op->perm.resize((size_t)N);
    std::iota(op->perm.begin(), op->perm.end(), 0);
    op->start.assign(1, 0);
    op->size.assign(1, (int32_t)N);
    op->parent.assign(1, -1);
    op->level.assign(1, 0);
    op->child0.clear();
    op->child1.clear();
    op->box.clear();
    std::vector<int32_t> scratch((size_t)N);

    for (size_t c = 0; c < op->start.size(); ++c) {
        const int32_t st = op->start[c], sz = op->size[c];
        // support box
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
        for (int32_t q = st; q < st + sz; ++q) {
            const int32_t i = op->perm[q];
            for (int64_t p = g->adj_ptr[i]; p < g->adj_ptr[i + 1]; ++p) {
                const int32_t* v = &g->tri[3 * (size_t)g->adj[p]];
                for (int a = 0; a < 3; ++a) {
                    const double* P = X + 3 * (int64_t)v[a];
                    for (int d = 0; d < 3; ++d) {
                        lo[d] = std::min(lo[d], P[d]);
                        hi[d] = std::max(hi[d], P[d]);
                    }
                }
            }
        }
        double longest = 0.0;
        for (int d = 0; d < 3; ++d) longest = std::max(longest, hi[d] - lo[d]);
        const double minw = rho * longest;
        for (int d = 0; d < 3; ++d) {
            if (hi[d] - lo[d] < minw) {
                const double cen = 0.5 * (lo[d] + hi[d]);
                lo[d] = cen - 0.5 * minw;
                hi[d] = cen + 0.5 * minw;
            }
        }
        for (int d = 0; d < 3; ++d) op->box.push_back(lo[d]);
        for (int d = 0; d < 3; ++d) op->box.push_back(hi[d]);
        op->child0.push_back(-1);
        op->child1.push_back(-1);
        if (sz <= leaf) continue;

        double nlo[3], nhi[3];
        for (int d = 0; d < 3; ++d) { nlo[d] = INFINITY; nhi[d] = -INFINITY; }
        for (int32_t q = st; q < st + sz; ++q) {
            const double* P = X + 3 * (int64_t)op->perm[q];
            for (int d = 0; d < 3; ++d) {
                nlo[d] = std::min(nlo[d], P[d]);
                nhi[d] = std::max(nhi[d], P[d]);
            }
        }
        int axis = 0;
        for (int d = 1; d < 3; ++d)
            if (nhi[d] - nlo[d] > nhi[axis] - nlo[axis]) axis = d;
        const double mid = (nlo[axis] + nhi[axis]) / 2.0;
        int32_t* lowp = scratch.data();
        int32_t nlow = 0, nhigh = 0;
        std::vector<int32_t> high;
        high.reserve((size_t)sz);
        for (int32_t q = st; q < st + sz; ++q) {
            const int32_t i = op->perm[q];
            if (X[3 * (int64_t)i + axis] <= mid) lowp[nlow++] = i;
            else { high.push_back(i); ++nhigh; }
        }
        if (nlow == 0 || nhigh == 0) continue;   // coincident nodes: stays a leaf
        std::memcpy(&op->perm[st], lowp, sizeof(int32_t) * nlow);
        std::memcpy(&op->perm[st + nlow], high.data(), sizeof(int32_t) * nhigh);
        const int32_t c0 = (int32_t)op->start.size();
        op->child0[c] = c0;
        op->child1[c] = c0 + 1;
        op->start.push_back(st);
        op->size.push_back(nlow);
        op->start.push_back(st + nlow);
        op->size.push_back(nhigh);
        for (int h = 0; h < 2; ++h) {
            op->parent.push_back((int32_t)c);
            op->level.push_back(op->level[c] + 1);
        }
    }
    op->nc = (int)op->start.size();
    op->nlevels = 1 + *std::max_element(op->level.begin(), op->level.end());
    op->nleaves = 0;
    for (int c = 0; c < op->nc; ++c) op->nleaves += op->child0[c] < 0;
}

namespace {
double diameter(const double* b) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) s += (b[3 + d] - b[d]) * (b[3 + d] - b[d]);
    return std::sqrt(s);
}
double distance(const double* a, const double* b) {
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
        double gap = 0.0;
        if (b[d] > a[3 + d]) gap = b[d] - a[3 + d];
        else if (a[d] > b[3 + d]) gap = a[d] - b[3 + d];
        s += gap * gap;
    }
    return std::sqrt(s);
}
}  // namespace

// Block partition: starting from (root, root), an admissible pair
// (max(diam B_t, diam B_s) <= eta dist(B_t, B_s)) becomes a far block, a pair
// of leaves a near block, anything else is refined into children(t) x
// children(s) with a leaf standing for itself.
void build_block_partition(h2_handle* op) {
    const double eta = op->params.eta;
    op->far_t.clear(); op->far_s.clear(); op->near_t.clear(); op->near_s.clear();
    std::vector<std::pair<int32_t, int32_t>> work{{0, 0}};
    while (!work.empty()) {
        auto [t, s] = work.back();
        work.pop_back();
        const double* bt = &op->box[6 * (size_t)t];
        const double* bs = &op->box[6 * (size_t)s];
        const double dmax = std::max(diameter(bt), diameter(bs));
        if (dmax <= eta * distance(bt, bs)) {
            op->far_t.push_back(t);
            op->far_s.push_back(s);
            continue;
        }
        const bool lt = op->child0[t] < 0, ls = op->child0[s] < 0;
        if (lt && ls) {
            op->near_t.push_back(t);
            op->near_s.push_back(s);
            continue;
        }
        int32_t ct[2] = {t, t}, cs[2] = {s, s};
        int nt = 1, ns = 1;
        if (!lt) { ct[0] = op->child0[t]; ct[1] = op->child1[t]; nt = 2; }
        if (!ls) { cs[0] = op->child0[s]; cs[1] = op->child1[s]; ns = 2; }
        for (int a = 0; a < nt; ++a)
            for (int b = 0; b < ns; ++b) work.emplace_back(ct[a], cs[b]);
    }
}

// Gauss-Legendre nodes and weights on [0, 1] (roots of P_q by Newton's method
// from the Tricomi-type initial guess cos(pi (i - 1/4)/(q + 1/2))).
void gauss_legendre_unit(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign((size_t)q, 0.0);
    w.assign((size_t)q, 0.0);
    for (int i = 1; i <= q; ++i) {
        double z = std::cos(M_PI * (i - 0.25) / (q + 0.5));
        double deriv = 1.0;
        for (int iter = 0; iter < 64; ++iter) {
            double pm1 = 0.0, p = 1.0;   // P_{-1} = 0, P_0 = 1
            for (int n = 1; n <= q; ++n) {
                const double pn = ((2 * n - 1) * z * p - (n - 1) * pm1) / n;
                pm1 = p;
                p = pn;
            }
            deriv = q * (pm1 - z * p) / (1.0 - z * z);
            const double step = p / deriv;
            z -= step;
            if (std::fabs(step) <= 1e-16) break;
        }
        x[(size_t)i - 1] = 0.5 * (1.0 - z);
        w[(size_t)i - 1] = 1.0 / ((1.0 - z * z) * deriv * deriv);
    }
}

}  // namespace h2
