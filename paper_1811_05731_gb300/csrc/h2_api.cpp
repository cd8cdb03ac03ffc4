// C ABI of the h2bem library (declared in include/h2bem.h).  Argument checks,
// handle life cycle and host <-> device staging; the numeric work is in
// h2_assemble.cu and h2_matvec.cu.
#include <atomic>
#include <chrono>
#include <cstring>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "h2_internal.h"

namespace h2 {
static thread_local std::string g_last_error;
void set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }
void set_cuda_error(cudaError_t e, const char* call, const char* file, int line) {
    const char* base = std::strrchr(file, '/');
    g_last_error = std::string(cudaGetErrorString(e)) + " (" + (base ? base + 1 : file) + ":" +
                   std::to_string(line) + ": " + call + ")";
}
}  // namespace h2

namespace {

// One NVTX range per public call (a no-op unless a profiler is attached), so
// that a timeline shows assembly, tuning and every product by name.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

void free_device(h2_handle* h) {
    auto f = [](void* p) {
        if (p) cudaFree(p);
    };
    if (h->kind == 1) {
        f(h->d_xyz); f(h->d_tri); f(h->d_adj_ptr); f(h->d_adj); f(h->d_psi);
    } else if (h->kind == 3) {
        h2::fem_release(h->fem);
        h->fem = nullptr;
    } else {
        h2::release_graph(h);
        if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
        h2::release_profile(h);
        for (h2::Pass& p : h->passes) { f(p.d_seg); f(p.d_chunk); f(p.d_piece); }
        f(h->d_arena); f(h->d_perm); f(h->d_box); f(h->d_ws); f(h->d_ws32); f(h->d_gather_src);
        f(h->d_zero_rows); f(h->d_io); f(h->d_err);
        f(h->d_fseg); f(h->d_fchunk); f(h->d_fpiece); f(h->d_fdeps); f(h->d_fexpect); f(h->d_fzero_rows);
        f(h->d_fcnt);
        f(h->d_sseg); f(h->d_schunk); f(h->d_spiece); f(h->d_sdeps); f(h->d_sexpect); f(h->d_szero_rows);
        f(h->d_u2n); f(h->d_near_units); f(h->d_nodes); f(h->d_near_pair); f(h->d_wsp);
        if (h->near_stream) cudaStreamDestroy(h->near_stream);
        if (h->ev_fork) cudaEventDestroy(h->ev_fork);
        if (h->ev_join) cudaEventDestroy(h->ev_join);
        delete h->rc;
        h->rc = nullptr;
    }
}

void release(h2_handle* h) {
    if (!h) return;
    if (--h->refcount > 0) return;
    h2_handle* g = h->kind == 2 ? h->geom : nullptr;
    free_device(h);
    delete h;
    if (g) release(g);
}

bool is_device_pointer(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

void h2_default_params(h2_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->m = 4;
    p->leaf = 64;
    p->eta = 2.0;
    p->box_inflation = 0.25;
    p->precision = H2_FP64;
    p->max_rhs = 1;
    p->schedule = H2_SCHEDULE_FLOW;
}

const char* h2_error_string(int code) {
    switch (code) {
        case H2_OK: return "ok";
        case H2_ERR_INVALID_ARG: return "invalid argument";
        case H2_ERR_MESH_OPEN: return "mesh is not a closed 2-manifold";
        case H2_ERR_MESH_ORIENTATION: return "mesh orientation is inconsistent or inward";
        case H2_ERR_DEGENERATE_TRIANGLE: return "degenerate triangle";
        case H2_ERR_OOM: return "out of memory";
        case H2_ERR_CUDA: return "CUDA error";
        case H2_ERR_TIMEOUT: return "device-side wait timed out";
        case H2_ERR_RHS_EXCEEDS_MAX: return "number of right-hand sides exceeds max_rhs";
        case H2_ERR_WRONG_HANDLE: return "wrong handle kind";
        case H2_ERR_SCRATCH_LIMIT: return "problem exceeds the fixed scratch of h2_matvec_noalloc";
        default: return "unknown status";
    }
}

const char* h2_last_error_message(void) { return h2::g_last_error.c_str(); }

int h2_build_geometry(const double* xyz, int64_t n_vertices, const int32_t* tri, int64_t n_triangles,
                      void* cuda_stream, h2_handle** out_geom) {
    if (!xyz || !tri || !out_geom) return H2_ERR_INVALID_ARG;
    *out_geom = nullptr;
    h2_handle* g = new (std::nothrow) h2_handle();
    if (!g) return H2_ERR_OOM;
    g->kind = 1;
    int rc = h2::validate_mesh(xyz, n_vertices, tri, n_triangles, g->adj_ptr, g->adj);
    if (rc != H2_OK) {
        delete g;
        return rc;
    }
    g->N = n_vertices;
    g->T = n_triangles;
    g->xyz.assign(xyz, xyz + 3 * n_vertices);
    g->tri.assign(tri, tri + 3 * n_triangles);
    cudaGetDevice(&g->device);
    rc = h2::geometry_device_setup(g, (cudaStream_t)cuda_stream);
    if (rc != H2_OK) {
        free_device(g);
        delete g;
        return rc;
    }
    *out_geom = g;
    return H2_OK;
}

int h2_assemble(const h2_handle* geom_c, const h2_params* p_in, h2_handle** out_op) {
    const Range range("h2_assemble");
    if (!geom_c || !out_op) return H2_ERR_INVALID_ARG;
    *out_op = nullptr;
    if (geom_c->kind != 1) return H2_ERR_WRONG_HANDLE;
    h2_params p;
    if (p_in) p = *p_in;
    else h2_default_params(&p);
    if (p.m < 1 || p.m > H2_MAX_M || p.leaf < 1 || p.leaf > H2_MAX_LEAF || !(p.eta > 0.0) ||
        !(p.box_inflation > 0.0) || p.box_inflation > 1.0 || p.max_rhs < 1 || p.max_rhs > H2_MAX_RHS ||
        p.precision < H2_FP64 || p.precision > H2_BF16X3 ||
        (p.schedule != H2_SCHEDULE_FLOW && p.schedule != H2_SCHEDULE_LEVELS))
        return H2_ERR_INVALID_ARG;
    if (p.autotune != 0 && p.autotune != 1) return H2_ERR_INVALID_ARG;
    if (p.coupling != H2_COUPLING_STORED && p.coupling != H2_COUPLING_ON_THE_FLY) return H2_ERR_INVALID_ARG;
    if (p.coupling == H2_COUPLING_ON_THE_FLY && p.precision != H2_FP32) return H2_ERR_INVALID_ARG;
    if (p.near_field != H2_NEAR_FP64 && p.near_field != H2_NEAR_F32PAIR) return H2_ERR_INVALID_ARG;
    if (p.near_field == H2_NEAR_F32PAIR &&
        ((p.precision != H2_FP32 && p.precision != H2_BF16X3) || p.max_rhs <= 8))
        return H2_ERR_INVALID_ARG;
    if (!(p.recompress_eps >= 0.0) || !(p.recompress_eps < 1.0) ||
        (p.recompress_eps > 0.0 && p.coupling != H2_COUPLING_STORED))
        return H2_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    h2_handle* geom = const_cast<h2_handle*>(geom_c);
    h2_handle* op = new (std::nothrow) h2_handle();
    if (!op) return H2_ERR_OOM;
    static std::atomic<uint64_t> next_serial{1};
    op->serial = next_serial++;
    op->kind = 2;
    op->geom = geom;
    geom->refcount++;
    op->params = p;
    op->m = p.m;
    op->k = p.m * p.m * p.m;
    op->kp = (op->k + 3) / 4 * 4;
    op->device = geom->device;
    h2::build_cluster_tree(op);
    h2::build_block_partition(op);
    int rc = H2_OK;
    if (p.recompress_eps > 0.0) {   // ranks per cluster before the product's layout
        rc = h2::recompress_device(op, nullptr);
        if (rc != H2_OK) {
            release(op);
            return rc;
        }
    }
    h2::build_plan(op);
    if (p.schedule == H2_SCHEDULE_FLOW || p.autotune) {   // the autotuner may pick either schedule
        h2::FlowModel fm;
        rc = h2::flow_model(op, fm);
        if (rc == H2_OK) op->flow_makespan_us = h2::build_flow(op, fm);
        if (rc == H2_OK && op->use_flow) rc = h2::build_split(op);
        if (p.schedule == H2_SCHEDULE_LEVELS) op->use_flow = 0;
    }
    if (rc == H2_OK) rc = h2::upload_plan(op);
    if (rc == H2_OK) rc = h2::assemble_device(op, nullptr);
    if (op->rc) op->rc->release_device();   // the ranks stay for h2_stats
    if (rc != H2_OK) {
        release(op);
        return rc;
    }
    if (p.autotune) {
        rc = h2::autotune(op, p.max_rhs, nullptr, nullptr);
        if (rc != H2_OK) {
            release(op);
            return rc;
        }
    }
    op->assemble_seconds =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out_op = op;
    return H2_OK;
}

int h2_fault_inject_stall(h2_handle* op, int32_t enable) {
    if (!op) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    if (!op->use_flow || !op->d_fexpect) return H2_ERR_INVALID_ARG;
    // the first region any segment of the ticket order waits for
    int32_t reg = -1;
    for (const h2::FlowSeg& f : op->fseg)
        if (f.ndep > 0) {
            reg = op->fdeps[f.dep0];
            break;
        }
    if (reg < 0) return H2_ERR_INVALID_ARG;
    const int32_t v = op->fexpect[reg] + (enable ? 1 : 0);   // one signal more than ever arrives
    H2_CUDA_TRY(cudaDeviceSynchronize());
    H2_CUDA_TRY(cudaMemcpy(op->d_fexpect + reg, &v, sizeof(int32_t), cudaMemcpyHostToDevice));
    return H2_OK;
}

int h2_autotune(h2_handle* op, int32_t r, void* cuda_stream, h2_tuning_t* out) {
    const Range range("h2_autotune");
    if (!op) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    if (r < 1 || r > op->params.max_rhs) return H2_ERR_INVALID_ARG;
    return h2::autotune(op, r, (cudaStream_t)cuda_stream, out);
}

int h2_matvec(h2_handle* op, const double* u1, double* u2, int32_t r, void* cuda_stream) {
    const Range range("h2_matvec");
    if (!op || !u1 || !u2) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    if (r < 1) return H2_ERR_INVALID_ARG;
    if (r > op->params.max_rhs) return H2_ERR_RHS_EXCEEDS_MAX;
    const int64_t N = op->geom->N;
    const size_t bytes = sizeof(double) * (size_t)N * r;
    const char *a = (const char*)u1, *b = (const char*)u2;
    if (a < b + bytes && b < a + bytes) return H2_ERR_INVALID_ARG;   // overlap
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const bool dev1 = is_device_pointer(u1), dev2 = is_device_pointer(u2);
    if (dev1 != dev2) return H2_ERR_INVALID_ARG;
    if (dev1) return h2::matvec_device(op, u1, u2, r, s);
    // host buffers: stage through device memory, synchronous
    if (!op->d_io) H2_CUDA_TRY(cudaMalloc((void**)&op->d_io, 2 * sizeof(double) * (size_t)N * op->params.max_rhs));
    double* d1 = op->d_io;
    double* d2 = op->d_io + (size_t)N * op->params.max_rhs;
    H2_CUDA_TRY(cudaMemcpyAsync(d1, u1, bytes, cudaMemcpyHostToDevice, s));
    int rc = h2::matvec_device(op, d1, d2, r, s);
    if (rc != H2_OK) return rc;
    H2_CUDA_TRY(cudaMemcpyAsync(u2, d2, bytes, cudaMemcpyDeviceToHost, s));
    H2_CUDA_TRY(cudaStreamSynchronize(s));
    int err = 0;
    H2_CUDA_TRY(cudaMemcpy(&err, op->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return err ? H2_ERR_TIMEOUT : H2_OK;
}

int h2_device_status(h2_handle* op) {
    if (!op) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    int err = 0;
    H2_CUDA_TRY(cudaDeviceSynchronize());
    H2_CUDA_TRY(cudaMemcpy(&err, op->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        H2_CUDA_TRY(cudaMemset(op->d_err, 0, sizeof(int)));
        return H2_ERR_TIMEOUT;
    }
    return H2_OK;
}

int h2_profile_enable(h2_handle* op, int32_t enable) {
    if (!op) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    std::vector<h2::ProfLaunch> launches;
    std::vector<double> ms;
    int n = 0;
    int rc = h2::read_profile(op, launches, ms, n);   // drops what was recorded so far
    if (rc != H2_OK) return rc;
    op->prof_enabled = enable ? 1 : 0;
    return H2_OK;
}

int h2_profile_read(h2_handle* op, int32_t capacity, int32_t* kind, double* ms_total, int64_t* bytes,
                    int64_t* macs, int32_t* grid, int32_t* n_calls, int32_t* n_entries) {
    if (!op || !n_calls || !n_entries) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    std::vector<h2::ProfLaunch> launches;
    std::vector<double> ms;
    int n = 0;
    int rc = h2::read_profile(op, launches, ms, n);
    if (rc != H2_OK) return rc;
    *n_calls = n;
    *n_entries = (int32_t)ms.size();
    for (int32_t i = 0; i < (int32_t)ms.size() && i < capacity; ++i) {
        const h2::ProfLaunch& L = launches[(size_t)i];
        if (kind) kind[i] = L.kind;
        if (ms_total) ms_total[i] = ms[(size_t)i];
        if (bytes) bytes[i] = L.bytes;
        if (macs) macs[i] = L.macs;
        if (grid) grid[i] = L.grid;
    }
    return H2_OK;
}

int h2_stats(const h2_handle* op, h2_stats_t* out) {
    if (!op || !out) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    std::memset(out, 0, sizeof(*out));
    const int64_t N = op->geom->N;
    out->n_vertices = N;
    out->n_triangles = op->geom->T;
    out->n_clusters = op->nc;
    out->n_levels = op->nlevels;
    out->n_leaves = op->nleaves;
    out->k = op->k;
    out->n_far_blocks = (int64_t)op->far_t.size();
    out->n_near_blocks = (int64_t)op->near_t.size();
    out->near_entries = op->near_entries;
    out->far_coefficients = (int64_t)op->far_t.size() * op->k * op->k;
    out->recompress_eps = op->params.recompress_eps;
    out->mean_rank_row = out->mean_rank_col = op->k;
    out->max_rank = op->k;
    if (op->rc) {
        out->far_coefficients = 0;
        for (size_t b = 0; b < op->far_t.size(); ++b)
            out->far_coefficients += (int64_t)op->rc->kr[op->far_t[b]] * op->rc->kc[op->far_s[b]];
        double sr = 0.0, sc = 0.0;
        int64_t nr = 0, ncn = 0;
        out->max_rank = 0;
        for (int c = 0; c < op->nc; ++c) {
            if (op->need_y[c]) {
                sr += op->rc->kr[c];
                ++nr;
            }
            if (op->need_x[c]) {
                sc += op->rc->kc[c];
                ++ncn;
            }
            out->max_rank = std::max(out->max_rank, std::max(op->rc->kr[c], op->rc->kc[c]));
        }
        out->mean_rank_row = nr ? sr / nr : 0.0;
        out->mean_rank_col = ncn ? sc / ncn : 0.0;
    }
    out->basis_coefficients = op->basis_coefficients;
    out->bytes_far = op->far_bytes;
    out->bytes_near = op->near_bytes;
    out->bytes_streamed = op->bytes_streamed;
    out->macs_per_rhs = op->macs;
    out->compression_ratio = 1.0 - (double)op->arena_bytes / (8.0 * (double)N * (double)N);
    out->assemble_seconds = op->assemble_seconds;
    out->precision = op->params.precision;
    out->max_rhs = op->params.max_rhs;
    out->n_launches_matvec = op->n_launches;
    out->n_passes = (int32_t)op->passes.size();
    out->bytes_near_pair = op->d_near_pair ? op->near_hi - op->near_lo : 0;
    out->near_field = op->params.near_field;
    out->coupling = op->params.coupling;
    return H2_OK;
}

int h2_get_tree(const h2_handle* op, int32_t* perm, int32_t* start, int32_t* size, int32_t* parent,
                int32_t* child0, int32_t* child1, int32_t* level, double* box) {
    if (!op) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    auto cp = [](void* dst, const void* src, size_t n) {
        if (dst) std::memcpy(dst, src, n);
    };
    cp(perm, op->perm.data(), sizeof(int32_t) * op->perm.size());
    cp(start, op->start.data(), sizeof(int32_t) * op->nc);
    cp(size, op->size.data(), sizeof(int32_t) * op->nc);
    cp(parent, op->parent.data(), sizeof(int32_t) * op->nc);
    cp(child0, op->child0.data(), sizeof(int32_t) * op->nc);
    cp(child1, op->child1.data(), sizeof(int32_t) * op->nc);
    cp(level, op->level.data(), sizeof(int32_t) * op->nc);
    cp(box, op->box.data(), sizeof(double) * 6 * op->nc);
    return H2_OK;
}

int h2_get_blocks(const h2_handle* op, int32_t* far_t, int32_t* far_s, int32_t* near_t, int32_t* near_s) {
    if (!op) return H2_ERR_INVALID_ARG;
    if (op->kind != 2) return H2_ERR_WRONG_HANDLE;
    auto cp = [](int32_t* dst, const std::vector<int32_t>& v) {
        if (dst && !v.empty()) std::memcpy(dst, v.data(), sizeof(int32_t) * v.size());
    };
    cp(far_t, op->far_t);
    cp(far_s, op->far_s);
    cp(near_t, op->near_t);
    cp(near_s, op->near_s);
    return H2_OK;
}

int h2_get_psi(const h2_handle* h, double* psi) {
    if (!h || !psi) return H2_ERR_INVALID_ARG;
    const h2_handle* g = h->kind == 2 ? h->geom : h;
    H2_CUDA_TRY(cudaMemcpy(psi, g->d_psi, sizeof(double) * g->N, cudaMemcpyDeviceToHost));
    return H2_OK;
}

int h2_free(h2_handle* h) {
    if (!h) return H2_OK;
    if (h->kind != 1 && h->kind != 2) return H2_ERR_WRONG_HANDLE;
    if (h->kind == 2) h2::drop_batch_plans(h->serial);
    release(h);
    return H2_OK;
}

int h2_matvec_batched(h2_handle* const* ops, int32_t n_ops, const double* const* u1, double* const* u2,
                      const int32_t* r, void* cuda_stream) {
    const Range range("h2_matvec_batched");
    if (!ops || !u1 || !u2 || !r || n_ops < 1 || n_ops > H2_MAX_BATCH) return H2_ERR_INVALID_ARG;
    for (int i = 0; i < n_ops; ++i) {
        if (!ops[i] || !u1[i] || !u2[i]) return H2_ERR_INVALID_ARG;
        if (ops[i]->kind != 2) return H2_ERR_WRONG_HANDLE;
        if (r[i] < 1) return H2_ERR_INVALID_ARG;
        if (r[i] > ops[i]->params.max_rhs) return H2_ERR_RHS_EXCEEDS_MAX;
        if (!is_device_pointer(u1[i]) || !is_device_pointer(u2[i])) return H2_ERR_INVALID_ARG;
        const size_t bytes = sizeof(double) * (size_t)ops[i]->geom->N * r[i];
        const char *a = (const char*)u1[i], *b = (const char*)u2[i];
        if (a < b + bytes && b < a + bytes) return H2_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ops[j] == ops[i]) return H2_ERR_INVALID_ARG;   // one workspace per operator
    }
    return h2::matvec_batched(ops, n_ops, u1, u2, r, (cudaStream_t)cuda_stream);
}

}  // extern "C"
