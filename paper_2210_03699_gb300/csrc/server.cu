// Request server with continuous batching over the multi-slot engine.
//
// Two host threads share one engine (fixed slot capacity):
//   setup thread: while a slot is free (running + ready + in setup < slots)
//      and the oldest waiting request fits the device-memory budget, set it
//      up on the GPU (tube, geometry, corrections, right-hand side, pair
//      schedules) on the handle's own stream and queue it as ready -- this
//      overlaps with the engine's steps instead of stalling them;
//   worker thread (owns the engine):
//   1. admit: put every ready handle into a free slot;
//   2. step: one engine step advances every admitted system (an Arnoldi
//      iteration, or a true-residual evaluation at a cycle end), so requests
//      that arrive while others run share the same launches;
//   3. retire: finished systems get their reaction potentials and energy,
//      their results are kept for the caller, their device memory is freed.
// Admission is first-come first-served: a request that does not fit waits
// for memory to free up (requests behind it wait too, so none starves).  The
// footprint estimate counts the tube nodes on the host (|d| < eps) and charges
// the per-node cost of geometry, packed sources, solver vectors and the
// Krylov basis plus the dense sum's exact node accumulators (200 bytes);
// after setup the handle's real allocation is charged instead.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "common.cuh"
#include "engine.cuh"

namespace ctr {

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    ctr_grid grid{};
    std::vector<double> sdist;
    double eps_in = 1, eps_out = 80, kappa = 0;
    std::vector<double> xyz, q;
    ctr_options opt{};
    ctr_request_result res{};
    std::vector<double> psi, dpsi;
    ctr_ibim* sys = nullptr;
    int slot = -1;
    int64_t need = 0;      // footprint estimate, computed at submission
    cudaStream_t stream = nullptr;   // the handle's own non-blocking stream (created and destroyed here)
    int64_t charged = 0;
    bool done = false;
    bool cancel = false;   // ctr_server_cancel: drop at the next point the owning thread reaches
};

size_t handle_bytes(const ctr_ibim* s) {
    const DevBuf* bufs[] = {&s->lin, &s->nodes, &s->src32, &s->src64, &s->srcdf, &s->corr_ptr, &s->corr_node,
                            &s->corr_w, &s->bad, &s->excl, &s->rhs, &s->charges, &s->acc, &s->err, &s->vecs,
                            &s->red, &s->map_ws, &s->map_io, &s->kr.V, &s->kr.H, &s->kr.cs, &s->kr.sn, &s->kr.s, &s->kr.y,
                            &s->kr.part, &s->kr.scal};
    size_t b = 0;
    for (const DevBuf* d : bufs) b += d->bytes;
    for (const PairSchedule& p : s->sched) b += p.d_items.bytes;
    b += s->counter.bytes;
    b += (size_t)tree_bytes(s);
    return b;
}

}  // namespace

}  // namespace ctr

struct ctr_server {
    int device = 0;
    int cap = 1;
    int64_t budget = 0;
    int64_t used = 0;
    int64_t peak_used = 0;
    int peak_slots = 0;
    ctr::Engine* engine = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ctr::Request*> waiting;
    std::deque<ctr::Request*> ready;     // set up, not yet in an engine slot
    int preparing = 0;                   // requests the setup thread is working on
    int admitting = 0;                   // set-up requests the worker has taken from `ready` to admit
    std::map<uint64_t, ctr::Request*> all;
    std::vector<ctr::Request*> running;
    uint64_t next_ticket = 1;
    bool stop = false;
    int fatal = 0;
    std::string fatal_msg;
    std::thread worker, setup;
    int64_t steps = 0;
};

namespace ctr {
namespace {

int64_t estimate_bytes(const Request& r) {
    const double eps = r.opt.tube_halfwidth > 0 ? r.opt.tube_halfwidth : 2.0 * r.grid.h;
    int64_t M = 0;
    for (double d : r.sdist) M += (std::fabs(d) < eps) ? 1 : 0;
    const int m = r.opt.restart > 0 ? r.opt.restart : 64;
    // per node: geometry 16 doubles, packed sources 64 + 64 + 64 bytes, corrections (~50 entries
    // worst case, K-reg) 36 bytes each, solver vectors 12 doubles, Krylov (m + 1) x 2 doubles, the
    // dense sum's exact accumulators 25 words; plus the pair schedules' items (a few MB)
    const int64_t per_node = 16 * 8 + 192 + 50 * 36 + 12 * 8 + (int64_t)(m + 1) * 16 + 25 * 8;
    // with the treecode: the tree-order exclusion lists, moment chunks and cluster charges
    const int64_t extra = (r.opt.farfield == CTR_FARFIELD_TREECODE) ? M * 512 + ((int64_t)64 << 20)
                                                                    : ((int64_t)16 << 20);
    const int64_t grid_bytes = (int64_t)r.sdist.size() * (8 + 4);   // staging copy + node map during setup
    return M * per_node + extra + grid_bytes;
}

void release_stream(Request* r) {
    if (r->stream) cudaStreamDestroy(r->stream);
    r->stream = nullptr;
}

void finish_request(ctr_server* sv, Request* r, int status) {
    r->res.status = status;
    r->res.t_done = now_s();
    r->done = true;
    sv->cv_done.notify_all();
}

// Retire the slots the last step finished (called with the lock released).
int retire_done(ctr_server* sv, const std::vector<SlotStat>& st, std::vector<Request*>& finished) {
    for (Request* r : sv->running) {
        if (st[r->slot].state != kSlotDone) continue;
        ctr_solve_info info{};
        const int rs = engine_retire(sv->engine, r->slot, &info);
        r->res.info = info;
        int status = rs < 0 ? rs : (info.converged ? CTR_OK : CTR_NOT_CONVERGED);
        const int64_t M = r->sys->M;
        r->res.M = M;
        if (status >= 0) {
            const double* x = r->sys->vecs.as<double>();
            r->psi.resize(M);
            r->dpsi.resize(M);
            if (cudaMemcpy(r->psi.data(), x, sizeof(double) * M, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(r->dpsi.data(), x + M, sizeof(double) * M, cudaMemcpyDeviceToHost) != cudaSuccess)
                status = fail(CTR_ERR_CUDA, "result copy");
        }
        if (status >= 0) {
            double G = 0.0;
            const int es = ctr_ibim_energy(r->sys, r->psi.data(), r->dpsi.data(), 0, &G, nullptr);
            if (es < 0) status = es;
            r->res.G_pol = G;
        }
        ctr_ibim_destroy(r->sys);
        r->sys = nullptr;
        release_stream(r);
        r->slot = -1;
        finished.push_back(r);
        r->res.status = status;
    }
    return CTR_OK;
}

// Setup thread: FCFS admission under the slot and memory limits, setup off the engine's thread.
void setup_loop(ctr_server* sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            auto can = [&] {
                if (sv->stop || sv->fatal) return true;
                if (sv->waiting.empty()) return false;
                const int in_flight = (int)(sv->running.size() + sv->ready.size()) + sv->preparing + sv->admitting;
                if (in_flight >= sv->cap) return false;
                // the oldest request goes in when it fits, or alone when it exceeds the budget
                return sv->used + sv->waiting.front()->need <= sv->budget || in_flight == 0;
            };
            sv->cv_work.wait(lk, can);
            if (sv->stop || sv->fatal) break;
            r = sv->waiting.front();
            sv->waiting.pop_front();
            r->charged = r->need;
            sv->used += r->need;
            sv->preparing++;
        }
        r->res.t_admit = now_s();
        ctr_ibim* sys = nullptr;
        // highest priority: setup kernels go ahead of the engine's queued ones between its launches
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        int s1 = (cudaStreamCreateWithPriority(&r->stream, cudaStreamNonBlocking, hi) == cudaSuccess)
                     ? CTR_OK
                     : fail(CTR_ERR_CUDA, "stream create");
        if (s1 >= 0)
            s1 = ctr_ibim_setup(&r->grid, r->sdist.data(), 0, r->eps_in, r->eps_out, r->kappa, (int64_t)r->q.size(),
                                r->xyz.data(), r->q.data(), &r->opt, r->stream, &sys);
        if (s1 < 0) {
            if (sys) ctr_ibim_destroy(sys);
            sys = nullptr;
            release_stream(r);
        }
        const int64_t real = sys ? (int64_t)handle_bytes(sys) : 0;
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->preparing--;
        r->sdist.clear();
        r->sdist.shrink_to_fit();
        if (s1 >= 0 && (sv->fatal || sv->stop)) {   // the engine is gone: nothing will run this system
            // free the system before the request is marked done (a waiter may release it at once)
            lk.unlock();
            ctr_ibim_destroy(sys);
            release_stream(r);
            lk.lock();
            sv->used -= r->charged;
            r->charged = 0;
            finish_request(sv, r, sv->fatal ? sv->fatal : CTR_ERR_INVALID);
            break;
        }
        if (s1 >= 0 && r->cancel) {   // cancelled during its setup
            lk.unlock();
            ctr_ibim_destroy(sys);
            release_stream(r);
            lk.lock();
            sv->used -= r->charged;
            r->charged = 0;
            finish_request(sv, r, CTR_ERR_CANCELLED);
        } else if (s1 < 0) {
            sv->used -= r->charged;
            r->charged = 0;
            finish_request(sv, r, s1);
        } else {
            // charge the real allocation instead of the estimate
            sv->used += real - r->charged;
            r->charged = real;
            r->sys = sys;
            sv->ready.push_back(r);
            sv->peak_used = std::max(sv->peak_used, sv->used);
        }
        sv->cv_work.notify_all();
    }
}

// Worker thread: owns the engine; admits ready systems, steps, retires.
void worker_loop(ctr_server* sv) {
    cudaSetDevice(sv->device);
    std::vector<SlotStat> st;
    for (;;) {
        std::deque<Request*> take;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->stop) break;
            if (sv->running.empty() && sv->ready.empty())
                sv->cv_work.wait(lk, [&] { return sv->stop || !sv->ready.empty(); });
            if (sv->stop) break;
            take.swap(sv->ready);
            sv->admitting = (int)take.size();   // still holding slots until admitted (or dropped)
        }
        for (Request* r : take) {
            bool cancelled;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                cancelled = r->cancel;
            }
            if (cancelled) {   // cancelled while set up and waiting for a slot
                ctr_ibim_destroy(r->sys);
                release_stream(r);
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->admitting--;
                r->sys = nullptr;
                sv->used -= r->charged;
                r->charged = 0;
                finish_request(sv, r, CTR_ERR_CANCELLED);
                sv->cv_work.notify_all();
                continue;
            }
            int slot = -1;
            const int s1 = engine_admit(sv->engine, r->sys, &slot);
            if (s1 < 0) {
                ctr_ibim_destroy(r->sys);
                release_stream(r);
            }
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->admitting--;
            if (s1 < 0) {
                r->sys = nullptr;
                sv->used -= r->charged;
                r->charged = 0;
                finish_request(sv, r, s1);
                sv->cv_work.notify_all();
            } else {
                r->slot = slot;
                sv->running.push_back(r);
                sv->peak_slots = std::max(sv->peak_slots, (int)sv->running.size());
            }
        }
        // cancelled running systems leave their slots between two steps
        std::vector<Request*> cancelled;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (Request* r : sv->running)
                if (r->cancel) cancelled.push_back(r);
        }
        for (Request* r : cancelled) {
            ctr_solve_info info{};
            (void)engine_retire(sv->engine, r->slot, &info);
            ctr_ibim_destroy(r->sys);
            release_stream(r);
            std::lock_guard<std::mutex> lk(sv->mu);
            r->sys = nullptr;
            r->slot = -1;
            r->res.info = info;
            sv->running.erase(std::find(sv->running.begin(), sv->running.end(), r));
            sv->used -= r->charged;
            r->charged = 0;
            finish_request(sv, r, CTR_ERR_CANCELLED);
            sv->cv_work.notify_all();
        }
        bool any;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            any = !sv->running.empty();
        }
        if (!any) continue;
        const int rs = engine_step(sv->engine, &st);
        std::vector<Request*> finished;
        if (rs < 0) {
            std::vector<Request*> drop;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->fatal = rs;
                sv->fatal_msg = ctr_last_error();
                for (Request* r : sv->running) {
                    finish_request(sv, r, rs);
                    drop.push_back(r);
                }
                sv->running.clear();
                for (Request* r : sv->ready) {
                    finish_request(sv, r, rs);
                    drop.push_back(r);
                }
                sv->ready.clear();
                for (Request* r : sv->waiting) finish_request(sv, r, rs);
                sv->waiting.clear();
                sv->cv_work.notify_all();   // the setup thread stops
            }
            for (Request* r : drop) {
                if (r->sys) ctr_ibim_destroy(r->sys);
                r->sys = nullptr;
                release_stream(r);
            }
            break;
        }
        retire_done(sv, st, finished);
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->steps++;
        for (Request* r : finished) {
            sv->running.erase(std::find(sv->running.begin(), sv->running.end(), r));
            sv->used -= r->charged;
            finish_request(sv, r, r->res.status);
        }
        if (!finished.empty()) sv->cv_work.notify_all();   // slots and memory were freed
    }
}

}  // namespace
}  // namespace ctr

using namespace ctr;

extern "C" {

void ctr_default_server_options(ctr_server_options* o) {
    if (!o) return;
    o->max_slots = 16;
    o->hbm_budget_bytes = 0;
    o->step_quantum_ms = 20.0;
}

int ctr_server_create(const ctr_server_options* opt, ctr_server** out) {
    if (!out) return fail(CTR_ERR_INVALID, "out is NULL");
    *out = nullptr;
    ctr_server_options o;
    ctr_default_server_options(&o);
    if (opt) o = *opt;
    if (o.max_slots <= 0 || o.max_slots > 4096) return fail(CTR_ERR_INVALID, "max_slots must be in [1, 4096]");
    if (!(o.step_quantum_ms >= 0.0 && o.step_quantum_ms <= 1e6))
        return fail(CTR_ERR_INVALID, "step_quantum_ms must be in [0, 1e6]");
    ctr_server* sv = new ctr_server();
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        delete sv;
        return fail(CTR_ERR_CUDA, "cudaGetDevice");
    }
    sv->cap = o.max_slots;
    if (o.hbm_budget_bytes > 0) {
        sv->budget = o.hbm_budget_bytes;
    } else {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete sv;
            return fail(CTR_ERR_CUDA, "cudaMemGetInfo");
        }
        sv->budget = (int64_t)(0.8 * (double)fr);
    }
    const int st = engine_create(sv->device, sv->cap, &sv->engine);
    if (st < 0) {
        delete sv;
        return st;
    }
    sv->engine->vec_blocks = 1;
    sv->engine->quantum_s = o.step_quantum_ms * 1e-3;
    sv->worker = std::thread(worker_loop, sv);
    sv->setup = std::thread(setup_loop, sv);
    *out = sv;
    return CTR_OK;
}

int ctr_server_submit(ctr_server* sv, const ctr_grid* grid, const double* sdist, double eps_in, double eps_out,
                      double kappa, int64_t n_charges, const double* charge_xyz, const double* charge_q,
                      const ctr_options* opt, uint64_t* ticket) {
    if (!sv || !grid || !sdist || !ticket || n_charges < 0 || (n_charges > 0 && (!charge_xyz || !charge_q)))
        return fail(CTR_ERR_INVALID, "bad argument");
    const int64_t total = grid->n[0] * grid->n[1] * grid->n[2];
    if (total <= 0) return fail(CTR_ERR_INVALID, "empty grid");
    Request* r = new Request();
    r->grid = *grid;
    r->sdist.assign(sdist, sdist + total);
    r->eps_in = eps_in;
    r->eps_out = eps_out;
    r->kappa = kappa;
    r->xyz.assign(charge_xyz ? charge_xyz : nullptr, charge_xyz ? charge_xyz + 3 * n_charges : nullptr);
    r->q.assign(charge_q ? charge_q : nullptr, charge_q ? charge_q + n_charges : nullptr);
    ctr_default_options(&r->opt);
    if (opt) r->opt = *opt;
    r->need = estimate_bytes(*r);   // outside the lock: it scans the grid
    r->res.t_submit = now_s();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal) {
        delete r;
        return fail(sv->fatal, "server stopped: " + sv->fatal_msg);
    }
    r->ticket = sv->next_ticket++;
    sv->all[r->ticket] = r;
    sv->waiting.push_back(r);
    *ticket = r->ticket;
    sv->cv_work.notify_all();   // both the setup thread and the worker wait on cv_work
    return CTR_OK;
}

int ctr_server_poll(ctr_server* sv, uint64_t ticket, int* done, ctr_request_result* res) {
    if (!sv || !done) return fail(CTR_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(CTR_ERR_INVALID, "unknown ticket");
    *done = it->second->done ? 1 : 0;
    if (*done && res) *res = it->second->res;
    return CTR_OK;
}

int ctr_server_wait(ctr_server* sv, uint64_t ticket, double timeout_s, ctr_request_result* res) {
    if (!sv) return fail(CTR_ERR_INVALID, "bad argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(CTR_ERR_INVALID, "unknown ticket");
    Request* r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_s > 0) {
        if (!sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
            return fail(CTR_ERR_DEVICE_WAIT, "timed out waiting for the request");
    } else {
        sv->cv_done.wait(lk, pred);
    }
    if (res) *res = r->res;
    return CTR_OK;
}

int ctr_server_fetch(ctr_server* sv, uint64_t ticket, double* psi, double* dpsi_n, int64_t capacity) {
    if (!sv) return fail(CTR_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(CTR_ERR_INVALID, "unknown ticket");
    Request* r = it->second;
    if (!r->done) return fail(CTR_ERR_INVALID, "request not finished");
    const int64_t M = (int64_t)r->psi.size();
    if (capacity < M) return fail(CTR_ERR_CAPACITY, "output buffers too small");
    if (psi) std::memcpy(psi, r->psi.data(), sizeof(double) * M);
    if (dpsi_n) std::memcpy(dpsi_n, r->dpsi.data(), sizeof(double) * M);
    return CTR_OK;
}

int ctr_server_release(ctr_server* sv, uint64_t ticket) {
    if (!sv) return fail(CTR_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(CTR_ERR_INVALID, "unknown ticket");
    if (!it->second->done) return fail(CTR_ERR_INVALID, "request not finished");
    delete it->second;
    sv->all.erase(it);
    return CTR_OK;
}

int ctr_server_cancel(ctr_server* sv, uint64_t ticket) {
    if (!sv) return fail(CTR_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->all.find(ticket);
    if (it == sv->all.end()) return fail(CTR_ERR_INVALID, "unknown ticket");
    Request* r = it->second;
    if (r->done) return fail(CTR_ERR_INVALID, "request already finished");
    auto q = std::find(sv->waiting.begin(), sv->waiting.end(), r);
    if (q != sv->waiting.end()) {   // still queued: nothing was charged or set up
        sv->waiting.erase(q);
        finish_request(sv, r, CTR_ERR_CANCELLED);
        return CTR_OK;
    }
    r->cancel = true;   // in setup, set up, or running: the owning thread drops it
    sv->cv_work.notify_all();
    return CTR_OK;
}

int ctr_server_stats(ctr_server* sv, ctr_server_stats_t* out) {
    if (!sv || !out) return fail(CTR_ERR_INVALID, "bad argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    out->budget_bytes = sv->budget;
    out->used_bytes = sv->used;
    out->peak_used_bytes = sv->peak_used;
    out->peak_slots = sv->peak_slots;
    out->running = (int)sv->running.size();
    out->waiting = (int)(sv->waiting.size() + sv->ready.size()) + sv->preparing + sv->admitting;
    out->steps = sv->steps;
    return CTR_OK;
}

void ctr_server_destroy(ctr_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->setup.joinable()) sv->setup.join();
    if (sv->worker.joinable()) sv->worker.join();
    for (std::vector<Request*> q : {sv->running, std::vector<Request*>(sv->ready.begin(), sv->ready.end())})
        for (Request* r : q) {
            if (r->sys) ctr_ibim_destroy(r->sys);
            r->sys = nullptr;
            release_stream(r);
        }
    for (auto& kv : sv->all) delete kv.second;
    delete sv->engine;
    delete sv;
}

}  // extern "C"
