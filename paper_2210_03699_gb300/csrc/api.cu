// C ABI entry points (declared in include/ctr_ibim.h): argument checks, handle
// lifetime, host/device staging.  No exception crosses this boundary.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "common.cuh"
#include "engine.cuh"

namespace ctr {

static thread_local std::string t_last_error;

void set_last_error(const std::string& msg) { t_last_error = msg; }

int fail(int status, const std::string& msg) {
    set_last_error(msg);
    return status;
}

static std::atomic<int64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace ctr

using namespace ctr;

namespace {

int copy_in(const double* src, int on_device, int64_t n, DevBuf& tmp, const double** out, cudaStream_t st) {
    if (on_device) {
        *out = src;
        return CTR_OK;
    }
    CTR_TRY(tmp.alloc(sizeof(double) * (n > 0 ? n : 1)));
    if (n > 0) CTR_CUDA_TRY(cudaMemcpyAsync(tmp.p, src, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    *out = tmp.as<double>();
    return CTR_OK;
}

int use_device(const ctr_ibim* s) {
    int cur = -1;
    CTR_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != s->device) CTR_CUDA_TRY(cudaSetDevice(s->device));
    return CTR_OK;
}

template <typename F>
int guarded(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return fail(CTR_ERR_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(CTR_ERR_INVALID, "unexpected internal exception");
    }
}

}  // namespace

extern "C" {

void ctr_default_options(ctr_options* o) {
    if (!o) return;
    o->tube_halfwidth = 0.0;
    o->precision = CTR_FP64;
    o->tol = 1e-10;
    o->restart = 64;
    o->max_iter = 400;
    o->max_refine = 10;
    o->inner_tol = 1e-5;
    o->tile_targets = 0;
    o->residual = CTR_DF64;
    o->method = CTR_METHOD_HYB;
    o->farfield = CTR_FARFIELD_DIRECT;
    o->tree_degree = 10;
    o->tree_theta = 0.8;
    o->tree_leaf = 128;
    o->tree_degree_fp32 = 6;
    o->tree_theta_fp32 = 0.9;
    o->residual_mode = CTR_RESIDUAL_UPDATE;
    o->fp32_block = 0;
    o->fp32_tile = 0;
}

const char* ctr_status_string(int st) {
    switch (st) {
        case CTR_OK: return "ok";
        case CTR_NOT_CONVERGED: return "not converged";
        case CTR_ERR_INVALID: return "invalid argument";
        case CTR_ERR_EMPTY_TUBE: return "empty tube";
        case CTR_ERR_GRID_MARGIN: return "tube node too close to the grid boundary";
        case CTR_ERR_CUDA: return "CUDA error";
        case CTR_ERR_NOMEM: return "out of device memory";
        case CTR_ERR_NUMERIC: return "non-finite value";
        case CTR_ERR_DEVICE_WAIT: return "bounded device wait expired";
        case CTR_ERR_CAPACITY: return "capacity exceeded";
        case CTR_ERR_CANCELLED: return "cancelled";
        default: return "unknown status";
    }
}

const char* ctr_last_error(void) { return t_last_error.c_str(); }

int64_t ctr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int ctr_tuning_info(int* targets_per_thread, int* chunk, int* unroll) {
    if (!targets_per_thread || !chunk || !unroll) return fail(CTR_ERR_INVALID, "NULL argument");
    const int v = last_fp32_variant();
    *targets_per_thread = v < 0 ? 0 : pk::kVar32[v].R * pk::Fp32x2Policy::kPack;
    *chunk = v < 0 ? 0 : pk::kVar32[v].V;
    *unroll = v < 0 ? 0 : pk::kVar32[v].U;
    return CTR_OK;
}

int ctr_ibim_pair_tuning(const ctr_ibim* s, int precision, int* block_targets, int* tile, int* chunk, int* unroll) {
    if (!s) return fail(CTR_ERR_INVALID, "NULL handle");
    if (precision != CTR_FP32_REFINE && precision != CTR_DF64 && precision != CTR_FP64)
        return fail(CTR_ERR_INVALID, "precision");
    const int pol = (precision == CTR_FP32_REFINE) ? 0 : (precision == CTR_DF64 ? 1 : 2);
    // an arithmetic the handle's options do not use is planned on first use (the handle's plan, not its state)
    CTR_TRY(ctr::ensure_schedule(const_cast<ctr_ibim*>(s), pol));
    const ctr::PairSchedule& p = s->sched[pol];
    if (block_targets) *block_targets = p.BS;
    if (tile) *tile = p.tile;
    if (chunk) *chunk = pol == 0 ? pk::kVar32[p.var].V : (pol == 1 ? pk::kChunkDf : pk::kChunk64);
    if (unroll) *unroll = pol == 0 ? pk::kVar32[p.var].U : 1;
    return CTR_OK;
}

void ctr_ibim_destroy(ctr_ibim* s) {
    if (!s) return;
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != s->device) cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    delete s;
    if (cur >= 0) cudaSetDevice(cur);
}

int ctr_ibim_setup(const ctr_grid* grid, const double* sdist, int sdist_on_device, double eps_in, double eps_out,
                   double kappa, int64_t n_charges, const double* charge_xyz, const double* charge_q,
                   const ctr_options* opt, void* stream, ctr_ibim** out) {
    return guarded([&]() -> int {
        if (!out) return fail(CTR_ERR_INVALID, "out is NULL");
        *out = nullptr;
        if (!grid || !sdist) return fail(CTR_ERR_INVALID, "grid or sdist is NULL");
        for (int c = 0; c < 3; ++c)
            if (grid->n[c] < 5) return fail(CTR_ERR_INVALID, "grid needs at least 5 nodes per axis");
        if (!(grid->h > 0.0) || !std::isfinite(grid->h)) return fail(CTR_ERR_INVALID, "grid spacing must be > 0");
        const int64_t total = grid->n[0] * grid->n[1] * grid->n[2];
        if (total > ((int64_t)1 << 31) - 1) return fail(CTR_ERR_CAPACITY, "grid larger than 2^31 nodes");
        if (!(eps_in > 0.0) || !(eps_out > 0.0) || !(kappa >= 0.0))
            return fail(CTR_ERR_INVALID, "eps_in, eps_out must be > 0 and kappa >= 0");
        if (n_charges < 0 || (n_charges > 0 && (!charge_xyz || !charge_q)))
            return fail(CTR_ERR_INVALID, "bad charges");
        for (int64_t c = 0; c < n_charges; ++c)
            if (!std::isfinite(charge_xyz[3 * c]) || !std::isfinite(charge_xyz[3 * c + 1]) ||
                !std::isfinite(charge_xyz[3 * c + 2]) || !std::isfinite(charge_q[c]))
                return fail(CTR_ERR_NUMERIC, "non-finite charge position or value");
        ctr_options o;
        ctr_default_options(&o);
        if (opt) {
            o = *opt;
            if (!(o.tol > 0)) o.tol = 1e-10;
            if (o.restart <= 0) o.restart = 64;
            if (o.max_iter <= 0) o.max_iter = 400;
            if (o.max_refine <= 0) o.max_refine = 10;
            if (!(o.inner_tol > 0)) o.inner_tol = 1e-5;
            if (o.precision != CTR_FP64 && o.precision != CTR_FP32_REFINE && o.precision != CTR_DF64)
                return fail(CTR_ERR_INVALID, "unknown precision");
            if (o.residual != CTR_FP64 && o.residual != CTR_DF64)
                return fail(CTR_ERR_INVALID, "residual must be CTR_FP64 or CTR_DF64");
            if (o.residual_mode != CTR_RESIDUAL_UPDATE && o.residual_mode != CTR_RESIDUAL_FULL)
                return fail(CTR_ERR_INVALID, "residual_mode must be CTR_RESIDUAL_UPDATE or CTR_RESIDUAL_FULL");
            if (o.method != CTR_METHOD_HYB && o.method != CTR_METHOD_KREG)
                return fail(CTR_ERR_INVALID, "method must be CTR_METHOD_HYB or CTR_METHOD_KREG");
            if (o.farfield != CTR_FARFIELD_DIRECT && o.farfield != CTR_FARFIELD_TREECODE)
                return fail(CTR_ERR_INVALID, "farfield must be CTR_FARFIELD_DIRECT or CTR_FARFIELD_TREECODE");
            if (o.tree_degree <= 0) o.tree_degree = 10;
            if (!(o.tree_theta > 0.0)) o.tree_theta = 0.8;
            if (o.tree_leaf <= 0) o.tree_leaf = 128;
            if (o.tree_degree_fp32 <= 0) o.tree_degree_fp32 = 6;
            if (!(o.tree_theta_fp32 > 0.0)) o.tree_theta_fp32 = 0.9;
            if (o.tree_degree < 2 || o.tree_degree > 12 || o.tree_degree_fp32 < 2 || o.tree_degree_fp32 > 12)
                return fail(CTR_ERR_INVALID, "tree degrees must be 2..12");
            if (!(o.tree_theta < 1.0) || !(o.tree_theta_fp32 < 1.0))
                return fail(CTR_ERR_INVALID, "tree theta must be below 1");
            if (o.tree_leaf > (1 << 20)) return fail(CTR_ERR_INVALID, "tree_leaf must be <= 2^20");
        }
        if (o.restart > 1000) return fail(CTR_ERR_INVALID, "restart must be <= 1000");
        ctr_ibim* s = new ctr_ibim();
        s->opt = o;
        CTR_CUDA_TRY(cudaGetDevice(&s->device));
        s->stream = static_cast<cudaStream_t>(stream);
        for (int c = 0; c < 3; ++c) {
            s->n[c] = grid->n[c];
            s->origin[c] = grid->origin[c];
        }
        s->h = grid->h;
        s->eps = (o.tube_halfwidth > 0.0) ? o.tube_halfwidth : 2.0 * grid->h;
        s->eps_in = eps_in;
        s->eps_out = eps_out;
        s->kappa = kappa;
        s->nc = n_charges;
        auto cleanup = [&](int st) {
            if (s->stream) cudaStreamSynchronize(s->stream);
            delete s;
            return st;
        };
        int st = s->err.alloc(sizeof(int));
        if (st < 0) return cleanup(st);
        if (cudaMemsetAsync(s->err.p, 0, sizeof(int), s->stream) != cudaSuccess)
            return cleanup(fail(CTR_ERR_CUDA, "memset"));
        DevBuf sd_tmp;
        const double* d_sd = nullptr;
        st = copy_in(sdist, sdist_on_device, total, sd_tmp, &d_sd, s->stream);
        if (st < 0) return cleanup(st);
        st = setup_tube_and_geometry(s, d_sd);
        if (st < 0) return cleanup(st);
        // charges as SoA x[nc], y[nc], z[nc], q[nc]
        std::vector<double> ch(4 * (size_t)std::max<int64_t>(n_charges, 1), 0.0);
        for (int64_t c = 0; c < n_charges; ++c) {
            ch[c] = charge_xyz[3 * c];
            ch[n_charges + c] = charge_xyz[3 * c + 1];
            ch[2 * n_charges + c] = charge_xyz[3 * c + 2];
            ch[3 * n_charges + c] = charge_q[c];
        }
        st = s->charges.alloc(sizeof(double) * ch.size());
        if (st < 0) return cleanup(st);
        if (cudaMemcpyAsync(s->charges.p, ch.data(), sizeof(double) * ch.size(), cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess)
            return cleanup(fail(CTR_ERR_CUDA, "charge upload"));
        st = setup_rhs(s);
        if (st < 0) return cleanup(st);
        st = plan_pairs(s);
        if (st < 0) return cleanup(st);
        st = s->vecs.alloc(sizeof(double) * 6 * 2 * (size_t)s->M);
        if (st < 0) return cleanup(st);
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) return cleanup(fail(CTR_ERR_CUDA, "setup sync"));
        st = check_device_error(s, "setup");
        if (st < 0) return cleanup(st);
        *out = s;
        return CTR_OK;
    });
}

int ctr_ibim_num_nodes(const ctr_ibim* s, int64_t* M) {
    if (!s || !M) return fail(CTR_ERR_INVALID, "NULL argument");
    *M = s->M;
    return CTR_OK;
}

int ctr_ibim_num_corrections(const ctr_ibim* s, int64_t* E) {
    if (!s || !E) return fail(CTR_ERR_INVALID, "NULL argument");
    *E = s->E;
    return CTR_OK;
}

int ctr_ibim_nodes(const ctr_ibim* s, int64_t* gi) {
    if (!s || !gi) return fail(CTR_ERR_INVALID, "NULL argument");
    CTR_TRY(use_device(s));
    CTR_CUDA_TRY(cudaMemcpyAsync(gi, s->lin.p, sizeof(int64_t) * s->M, cudaMemcpyDeviceToHost, s->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return CTR_OK;
}

int ctr_ibim_geometry(const ctr_ibim* s, double* P, double* normal, double* W) {
    if (!s) return fail(CTR_ERR_INVALID, "NULL handle");
    return guarded([&]() -> int {
        CTR_TRY(use_device(s));
        const int64_t M = s->M;
        std::vector<double> h(6 * (size_t)M + M);
        CTR_CUDA_TRY(cudaMemcpyAsync(h.data(), s->nodes.p, sizeof(double) * 7 * M, cudaMemcpyDeviceToHost, s->stream));
        CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
        for (int64_t m = 0; m < M; ++m) {
            if (P) {
                P[3 * m] = h[m];
                P[3 * m + 1] = h[M + m];
                P[3 * m + 2] = h[2 * M + m];
            }
            if (normal) {
                normal[3 * m] = h[3 * M + m];
                normal[3 * m + 1] = h[4 * M + m];
                normal[3 * m + 2] = h[5 * M + m];
            }
            if (W) W[m] = h[6 * M + m];
        }
        return CTR_OK;
    });
}

int ctr_ibim_corrections(const ctr_ibim* s, int64_t* ptr, int64_t* node, double* w11, double* w12, double* w21,
                         double* w22) {
    if (!s) return fail(CTR_ERR_INVALID, "NULL handle");
    return guarded([&]() -> int {
        CTR_TRY(use_device(s));
        const int64_t M = s->M, E = s->E;
        std::vector<int32_t> p(M + 1), nd(E);
        std::vector<double> w(4 * (size_t)E);
        CTR_CUDA_TRY(cudaMemcpyAsync(p.data(), s->corr_ptr.p, sizeof(int32_t) * (M + 1), cudaMemcpyDeviceToHost, s->stream));
        CTR_CUDA_TRY(cudaMemcpyAsync(nd.data(), s->corr_node.p, sizeof(int32_t) * E, cudaMemcpyDeviceToHost, s->stream));
        CTR_CUDA_TRY(cudaMemcpyAsync(w.data(), s->corr_w.p, sizeof(double) * 4 * E, cudaMemcpyDeviceToHost, s->stream));
        CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (ptr) for (int64_t i = 0; i <= M; ++i) ptr[i] = p[i];
        if (node) for (int64_t e = 0; e < E; ++e) node[e] = nd[e];
        if (w11) std::memcpy(w11, w.data(), sizeof(double) * E);
        if (w21) std::memcpy(w21, w.data() + E, sizeof(double) * E);
        if (w22) std::memcpy(w22, w.data() + 2 * E, sizeof(double) * E);
        if (w12) std::memcpy(w12, w.data() + 3 * E, sizeof(double) * E);
        return CTR_OK;
    });
}

int ctr_ibim_bad_nodes(const ctr_ibim* s, uint8_t* flags) {
    if (!s || !flags) return fail(CTR_ERR_INVALID, "NULL argument");
    CTR_TRY(use_device(s));
    CTR_CUDA_TRY(cudaMemcpyAsync(flags, s->bad.p, s->M, cudaMemcpyDeviceToHost, s->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return CTR_OK;
}

int ctr_ibim_rhs(const ctr_ibim* s, double* g, int on_device) {
    if (!s || !g) return fail(CTR_ERR_INVALID, "NULL argument");
    CTR_TRY(use_device(s));
    CTR_CUDA_TRY(cudaMemcpyAsync(g, s->rhs.p, sizeof(double) * 2 * s->M,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return CTR_OK;
}

int ctr_ibim_pair_schedule(const ctr_ibim* s, int precision, int64_t* one_sided, int64_t* symmetric,
                           int64_t* items, int64_t* partial_bytes) {
    if (!s) return fail(CTR_ERR_INVALID, "NULL handle");
    if (precision != CTR_FP32_REFINE && precision != CTR_DF64 && precision != CTR_FP64)
        return fail(CTR_ERR_INVALID, "precision");
    const int pol = (precision == CTR_FP32_REFINE) ? 0 : (precision == CTR_DF64 ? 1 : 2);
    // an arithmetic the handle's options do not use is planned on first use (the handle's plan, not its state)
    CTR_TRY(ctr::ensure_schedule(const_cast<ctr_ibim*>(s), pol));
    const ctr::PairSchedule& p = s->sched[pol];
    if (one_sided) *one_sided = p.pairs_one;
    if (symmetric) *symmetric = p.pairs_sym;
    if (items) *items = (int64_t)p.items.size();
    if (partial_bytes) *partial_bytes = (int64_t)s->acc.bytes;
    return CTR_OK;
}

int ctr_ibim_farfield_info(const ctr_ibim* s, int precision, int64_t* perm, int64_t* near_pairs,
                           int64_t* far_evaluations, int64_t* far_interactions, int64_t* far_clusters) {
    if (!s) return fail(CTR_ERR_INVALID, "NULL handle");
    if (!s->tree) return fail(CTR_ERR_INVALID, "handle was set up without the treecode");
    if (precision != CTR_FP32_REFINE && precision != CTR_DF64 && precision != CTR_FP64)
        return fail(CTR_ERR_INVALID, "precision");
    const int pol = (precision == CTR_FP32_REFINE) ? 0 : (precision == CTR_DF64 ? 1 : 2);
    const ctr::TreeData& t = *s->tree;
    if (perm)
        for (int64_t p = 0; p < s->M; ++p) perm[p] = t.perm[(size_t)p];
    if (near_pairs) *near_pairs = t.pol[pol].near_pairs;
    if (far_evaluations) *far_evaluations = t.pol[pol].far_evals;
    if (far_interactions) *far_interactions = t.pol[pol].far_pairs;
    if (far_clusters) *far_clusters = t.pol[pol].nq;
    return CTR_OK;
}

int ctr_ibim_time_operator(ctr_ibim* s, int precision, int reps, double* pack_ms, double* pairs_ms,
                           double* far_ms, double* finish_ms) {
    return guarded([&]() -> int {
        if (!s) return fail(CTR_ERR_INVALID, "NULL handle");
        if (reps < 1) return fail(CTR_ERR_INVALID, "reps must be >= 1");
        if (precision != CTR_FP32_REFINE && precision != CTR_DF64 && precision != CTR_FP64)
            return fail(CTR_ERR_INVALID, "precision");
        CTR_TRY(use_device(s));
        const int64_t n = 2 * s->M;
        double* y = s->vecs.as<double>() + 5 * n;   // the last solver vector as scratch
        cudaEvent_t ev[5];
        for (auto& e : ev) CTR_CUDA_TRY(cudaEventCreate(&e));
        double acc[4] = {0, 0, 0, 0};
        int st = CTR_OK;
        for (int r = 0; r <= reps && st == CTR_OK; ++r) {   // the first application warms up
            st = apply_operator_timed(s, s->rhs.as<double>(), y, precision, ev);
            if (st == CTR_OK && cudaEventSynchronize(ev[4]) != cudaSuccess) st = fail(CTR_ERR_CUDA, "event sync");
            for (int k = 0; k < 4 && st == CTR_OK && r > 0; ++k) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) st = fail(CTR_ERR_CUDA, "event time");
                acc[k] += ms;
            }
        }
        for (auto& e : ev) cudaEventDestroy(e);
        CTR_TRY(st);
        CTR_TRY(check_device_error(s, "time_operator"));
        if (pack_ms) *pack_ms = acc[0] / reps;
        if (pairs_ms) *pairs_ms = acc[1] / reps;
        if (far_ms) *far_ms = acc[2] / reps;
        if (finish_ms) *finish_ms = acc[3] / reps;
        return CTR_OK;
    });
}

int ctr_ibim_area(const ctr_ibim* s, double* area) {
    if (!s || !area) return fail(CTR_ERR_INVALID, "NULL argument");
    return guarded([&]() -> int {
        CTR_TRY(use_device(s));
        std::vector<double> W(s->M);
        CTR_CUDA_TRY(cudaMemcpyAsync(W.data(), s->na.W, sizeof(double) * s->M, cudaMemcpyDeviceToHost, s->stream));
        CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
        double a = 0.0;
        for (double v : W) a += v;
        *area = a * s->h * s->h * s->h;
        return CTR_OK;
    });
}

int ctr_ibim_matvec(ctr_ibim* s, const double* x, double* y, int precision, int on_device) {
    if (!s || !x || !y) return fail(CTR_ERR_INVALID, "NULL argument");
    if (precision != CTR_FP64 && precision != CTR_FP32_REFINE && precision != CTR_DF64)
        return fail(CTR_ERR_INVALID, "unknown precision");
    return guarded([&]() -> int {
        CTR_TRY(use_device(s));
        const int64_t n = 2 * s->M;
        DevBuf xin, yout;
        const double* dx = nullptr;
        CTR_TRY(copy_in(x, on_device, n, xin, &dx, s->stream));
        double* dy = y;
        if (!on_device) {
            CTR_TRY(yout.alloc(sizeof(double) * n));
            dy = yout.as<double>();
        }
        CTR_TRY(apply_operator(s, dx, dy, precision));
        if (!on_device) CTR_CUDA_TRY(cudaMemcpyAsync(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
        CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
        return check_device_error(s, "matvec");
    });
}

int ctr_ibim_solve(ctr_ibim* s, double* psi, double* dpsi_n, int on_device, ctr_solve_info* info) {
    if (!s || !psi || !dpsi_n) return fail(CTR_ERR_INVALID, "NULL argument");
    ctr_ibim* hs[1] = {s};
    double* p[1] = {psi};
    double* d[1] = {dpsi_n};
    return ctr_ibim_batch_solve(hs, 1, p, d, on_device, info);
}

int ctr_ibim_batch_solve(ctr_ibim* const* systems, int64_t n, double* const* psi, double* const* dpsi_n,
                         int on_device, ctr_solve_info* infos) {
    if (n < 0 || (n > 0 && (!systems || !psi || !dpsi_n))) return fail(CTR_ERR_INVALID, "NULL argument");
    if (n == 0) return CTR_OK;
    return guarded([&]() -> int {
        for (int64_t i = 0; i < n; ++i) {
            if (!systems[i] || !psi[i] || !dpsi_n[i]) return fail(CTR_ERR_INVALID, "NULL system or output");
            if (systems[i]->device != systems[0]->device)
                return fail(CTR_ERR_INVALID, "all systems of a batch must be on one device");
            for (int64_t k = 0; k < i; ++k)
                if (systems[k] == systems[i]) return fail(CTR_ERR_INVALID, "a system appears twice in the batch");
        }
        CTR_TRY(use_device(systems[0]));
        std::vector<ctr_solve_info> local;
        int64_t steps = 0;
        const int st = engine_solve_all(systems, n, 1, &local, &steps);
        if (infos)
            for (int64_t i = 0; i < n && i < (int64_t)local.size(); ++i) infos[i] = local[i];
        if (st < 0) return st;
        bool all_conv = true;
        for (int64_t i = 0; i < n; ++i) {
            ctr_ibim* s = systems[i];
            const int64_t M = s->M;
            const double* x = s->vecs.as<double>();
            const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            CTR_CUDA_TRY(cudaMemcpyAsync(psi[i], x, sizeof(double) * M, kind, s->stream));
            CTR_CUDA_TRY(cudaMemcpyAsync(dpsi_n[i], x + M, sizeof(double) * M, kind, s->stream));
            CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
            all_conv &= (local[i].converged != 0);
        }
        return all_conv ? CTR_OK : CTR_NOT_CONVERGED;
    });
}

int ctr_ibim_reaction_potential(ctr_ibim* s, const double* psi, const double* dpsi_n, int on_device, int64_t n_points,
                                const double* xyz, double* out) {
    if (!s || !psi || !dpsi_n || (n_points > 0 && (!xyz || !out)) || n_points < 0)
        return fail(CTR_ERR_INVALID, "NULL argument");
    return guarded([&]() -> int {
        CTR_TRY(use_device(s));
        if (n_points == 0) return CTR_OK;
        // psi and dpsi where the caller has them; points and results staged in the handle's buffers
        const int64_t M = s->M;
        const int64_t need = (on_device ? 0 : 2 * M) + 4 * n_points;
        CTR_TRY(s->map_io.alloc(sizeof(double) * (size_t)need));
        double* io = s->map_io.as<double>();
        const double* dp = psi;
        const double* dd = dpsi_n;
        if (!on_device) {
            CTR_CUDA_TRY(cudaMemcpyAsync(io, psi, sizeof(double) * M, cudaMemcpyHostToDevice, s->stream));
            CTR_CUDA_TRY(cudaMemcpyAsync(io + M, dpsi_n, sizeof(double) * M, cudaMemcpyHostToDevice, s->stream));
            dp = io;
            dd = io + M;
            io += 2 * M;
        }
        CTR_CUDA_TRY(cudaMemcpyAsync(io, xyz, sizeof(double) * 3 * n_points, cudaMemcpyHostToDevice, s->stream));
        CTR_TRY(potential_map(s, dp, dd, n_points, io, io + 3 * n_points, CTR_FP64));
        CTR_CUDA_TRY(cudaMemcpyAsync(out, io + 3 * n_points, sizeof(double) * n_points, cudaMemcpyDeviceToHost,
                                     s->stream));
        CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
        return check_device_error(s, "reaction potential");
    });
}

int ctr_ibim_potential_map(ctr_ibim* s, const double* psi, const double* dpsi_n, int64_t n_points, const double* xyz,
                           double* out, int precision, int on_device) {
    if (!s || !psi || !dpsi_n || n_points < 0 || (n_points > 0 && (!xyz || !out)))
        return fail(CTR_ERR_INVALID, "NULL argument");
    if (precision != CTR_FP64 && precision != CTR_FP32_REFINE && precision != CTR_DF64)
        return fail(CTR_ERR_INVALID, "unknown precision");
    return guarded([&]() -> int {
        CTR_TRY(use_device(s));
        if (n_points == 0) return CTR_OK;
        if (on_device) {
            CTR_TRY(potential_map(s, psi, dpsi_n, n_points, xyz, out, precision));
            CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
            return check_device_error(s, "potential map");
        }
        const int64_t M = s->M;
        CTR_TRY(s->map_io.alloc(sizeof(double) * (size_t)(2 * M + 4 * n_points)));
        double* io = s->map_io.as<double>();
        CTR_CUDA_TRY(cudaMemcpyAsync(io, psi, sizeof(double) * M, cudaMemcpyHostToDevice, s->stream));
        CTR_CUDA_TRY(cudaMemcpyAsync(io + M, dpsi_n, sizeof(double) * M, cudaMemcpyHostToDevice, s->stream));
        CTR_CUDA_TRY(cudaMemcpyAsync(io + 2 * M, xyz, sizeof(double) * 3 * n_points, cudaMemcpyHostToDevice,
                                     s->stream));
        double* d_out = io + 2 * M + 3 * n_points;
        CTR_TRY(potential_map(s, io, io + M, n_points, io + 2 * M, d_out, precision));
        CTR_CUDA_TRY(cudaMemcpyAsync(out, d_out, sizeof(double) * n_points, cudaMemcpyDeviceToHost, s->stream));
        CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
        return check_device_error(s, "potential map");
    });
}

int ctr_ibim_energy(ctr_ibim* s, const double* psi, const double* dpsi_n, int on_device, double* G_pol,
                    double* psi_rxn) {
    if (!s || !psi || !dpsi_n || !G_pol) return fail(CTR_ERR_INVALID, "NULL argument");
    return guarded([&]() -> int {
        CTR_TRY(use_device(s));
        const int64_t nc = s->nc;
        *G_pol = 0.0;
        if (nc == 0) return CTR_OK;
        std::vector<double> ch(4 * (size_t)nc), xyz(3 * (size_t)nc), prx(nc);
        CTR_CUDA_TRY(cudaMemcpyAsync(ch.data(), s->charges.p, sizeof(double) * 4 * nc, cudaMemcpyDeviceToHost, s->stream));
        CTR_CUDA_TRY(cudaStreamSynchronize(s->stream));
        for (int64_t c = 0; c < nc; ++c) {
            xyz[3 * c] = ch[c];
            xyz[3 * c + 1] = ch[nc + c];
            xyz[3 * c + 2] = ch[2 * nc + c];
        }
        CTR_TRY(ctr_ibim_reaction_potential(s, psi, dpsi_n, on_device, nc, xyz.data(), prx.data()));
        double G = 0.0;
        for (int64_t c = 0; c < nc; ++c) G += ch[3 * nc + c] * prx[c];
        *G_pol = 0.5 * G;
        if (psi_rxn) std::memcpy(psi_rxn, prx.data(), sizeof(double) * nc);
        return CTR_OK;
    });
}

int ctr_weight_tables(double* out) {
    if (!out) return fail(CTR_ERR_INVALID, "NULL argument");
    DevBuf t;
    CTR_TRY(t.alloc(sizeof(double) * kTabSize));
    CTR_TRY(weight_tables_device(t.as<double>(), nullptr));
    CTR_CUDA_TRY(cudaMemcpy(out, t.p, sizeof(double) * kTabSize, cudaMemcpyDeviceToHost));
    return CTR_OK;
}

}  // extern "C"
