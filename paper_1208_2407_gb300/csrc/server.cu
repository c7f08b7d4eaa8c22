// Continuous-batching server for Trotter-Suzuki evolutions of many grids.
//
// Requests (a grid size, a potential, an initial state, dt, theta and a step
// count) arrive at any time.  A scheduler thread admits them in arrival order
// while device memory (the budget) and slots allow, uploads their inputs on a
// copy stream, and advances every admitted grid together: each epoch is a
// short run of launches of the multi-grid fused kernel (fused.cu), in which
// all runnable grids share the persistent warps, so their work overlaps on
// the GPU.  Requests that arrive while an epoch runs join at the next one.
// Each grid gets floor(steps/K) launches at depth K and one at depth
// steps % K, the same sequence as evolving it alone, so its result does not
// depend on the mix.  Finished states stay on the device until the client
// fetches and releases them.  Repeated epochs with the same launch shape run
// as cached CUDA graphs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/trotter.h"
#include "grid.h"
#include "internal.h"
#include "trace.h"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

ts_status err(ts_status s, const char *fmt, ...)
{
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return (ts_status)ts::set_error(s, "%s", buf);
}

enum ReqState { R_PENDING, R_ACTIVE, R_DONE, R_FAILED, R_CANCELLED };

struct Req {
    uint64_t ticket = 0;
    ts_request r{};
    size_t bytes = 0;
    ReqState state = R_PENDING;
    ts_status status = TS_OK;
    ts_grid *g = nullptr;
    void *slab = nullptr;
    cudaEvent_t ready = nullptr;    // inputs uploaded
    bool ready_seen = false;
    int64_t full_left = 0, rem_left = 0;   // launches still to enqueue
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    bool cancel = false;
    bool reserved = false;          // counted in the server's bytes in use
    int inflight = 0;               // queued epochs that include this request
    char why[160] = "";             // reason of a failure
};

void note(Req &q, const char *where, cudaError_t e)
{
    snprintf(q.why, sizeof(q.why), "%s: %s", where, cudaGetErrorString(e));
}
using ReqP = std::shared_ptr<Req>;

struct Epoch {
    cudaEvent_t done = nullptr;
    int *err_copy = nullptr;        // pinned host copy of the error word after this epoch
    std::vector<ReqP> members, finishing;
    std::vector<int> tables;
};

struct GraphKey {
    int slot, n, L, K;
    int warps;
    int64_t units;
    bool aligned;
    bool operator==(const GraphKey &o) const
    {
        return slot == o.slot && n == o.n && L == o.L && K == o.K && warps == o.warps &&
               units == o.units && aligned == o.aligned;
    }
};

constexpr int kTables = 32;

}  // namespace

struct ts_server {
    ts_server_cfg cfg{};
    int K = 4, L_max = 8;
    int device = 0;                 // the creating thread's device; the worker runs there
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, ReqP> reqs;
    std::deque<ReqP> pending;
    std::vector<ReqP> active;
    std::deque<Epoch> inflight;
    uint64_t next_ticket = 1;
    size_t used = 0, peak = 0;
    bool stop = false, dead = false;
    cudaStream_t compute = nullptr, copy = nullptr;
    int *err_host = nullptr, *err_dev = nullptr;   // kernel error word and its pinned copy
    ts::EpochEntry *tab_dev = nullptr, *tab_host = nullptr;
    cudaEvent_t tab_free[kTables] = {};
    int tab_next = 0;
    std::vector<std::pair<GraphKey, cudaGraphExec_t>> graphs;
    std::thread worker;
    // statistics
    std::vector<double> lat_ms;
    int64_t submitted = 0, completed = 0, failed = 0, epochs = 0, graph_launches = 0;
    double site_steps_done = 0.0;
    int64_t t_first = 0, t_last = 0;

    void run();
    bool admit_one(const ReqP &q);
    void enqueue_epoch(std::unique_lock<std::mutex> &lk);
    void retire(Epoch &e, bool ok);
    int take_table();
    cudaError_t launch_full(int slot, int n, const ts::MultiPlan &plan, int L);
};

int ts_server::take_table()
{
    const int s = tab_next;
    tab_next = (tab_next + 1) % kTables;
    cudaEventSynchronize(tab_free[s]);   // the epoch that last used this slot is done
    return s;
}

cudaError_t ts_server::launch_full(int slot, int n, const ts::MultiPlan &plan, int L)
{
    const ts::EpochEntry *tab = tab_dev + (size_t)slot * cfg.max_slots;
    if (L == 1) return ts::launch_fused_multi(K, tab, n, plan, 0, err_dev, compute);
    const GraphKey key{slot, n, L, K, plan.warps, plan.units, plan.aligned};
    for (auto &kv : graphs)
        if (kv.first == key) {
            ++graph_launches;
            ts::count_launches(L);
            return cudaGraphLaunch(kv.second, compute);
        }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(compute, cudaStreamCaptureModeThreadLocal);
    for (int t = 0; t < L && e == cudaSuccess; ++t)
        e = ts::launch_fused_multi(K, tab, n, plan, t & 1, err_dev, compute);
    cudaError_t e2 = cudaStreamEndCapture(compute, &graph);
    if (e == cudaSuccess) e = e2;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    if (graphs.size() >= 64) {
        cudaGraphExecDestroy(graphs.front().second);
        graphs.erase(graphs.begin());
    }
    graphs.push_back({key, exec});
    ++graph_launches;
    return cudaGraphLaunch(exec, compute);
}

// Allocate and fill one admitted request's grid on the copy stream.
bool ts_server::admit_one(const ReqP &q)
{
    ts::TraceRange trace_("server admit");
    const ts_request &r = q->r;
    ts_layout L;
    ts_grid_layout(r.nx, r.ny, TS_F32, &L);
    cudaError_t e = cudaMallocAsync(&q->slab, L.slab_bytes, copy);
    // the tensor-map encoder validates the address, so the stream-ordered
    // allocation must have happened before the grid is set up
    if (e == cudaSuccess) e = cudaStreamSynchronize(copy);
    if (e != cudaSuccess) {
        cudaGetLastError();
        note(*q, "slab allocation", e);
        q->status = TS_ERR_OOM;
        return false;
    }
    if (ts::grid_setup(L, q->slab, false, &q->g) != TS_OK) {
        snprintf(q->why, sizeof(q->why), "grid set-up: %s", ts_last_error());
        q->status = TS_ERR_CUDA;
        return false;
    }
    ts_grid *g = q->g;
    const int nx = (int)r.nx, ny = (int)r.ny;
    const size_t n = (size_t)nx * ny;
    const size_t scr = ts::grid_scratch_offset(L);
    e = cudaMemsetAsync(g->slab + scr, 0, L.slab_bytes - scr, copy);
    ts::grid_set_coefficients(g, r.dt, r.theta, copy);
    // potential -> tables (host input staged through the idle ping-pong pair)
    if (e == cudaSuccess && r.V) {
        const double *src = r.V;
        if (r.where == TS_HOST) {
            e = cudaMemcpyAsync(g->re_other(), r.V, n * 8, cudaMemcpyHostToDevice, copy);
            src = (const double *)g->re_other();
        }
        if (e == cudaSuccess)
            e = ts::launch_phase_table(src, g->pg(), g->ps(), g->vp(), false, nx, ny, L.pitch, r.dt,
                                       copy);
    } else if (e == cudaSuccess) {
        e = cudaMemsetAsync(g->pg(), 0, 3 * L.plane_bytes, copy);
    }
    // initial state
    const bool f64 = r.psi_dtype == TS_F64;
    const void *src[2] = {r.psi_re, r.psi_im};
    void *dst[2] = {g->re(), g->im()};
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
        const void *s = src[c];
        if (r.where == TS_HOST) {
            e = cudaMemcpyAsync(g->re_other(), s, n * (f64 ? 8 : 4), cudaMemcpyHostToDevice, copy);
            s = g->re_other();
        }
        if (e == cudaSuccess) e = ts::launch_convert_in(s, f64, dst[c], false, nx, ny, L.pitch, copy);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(q->ready, copy);
    if (e != cudaSuccess) {
        note(*q, "input upload", e);
        q->status = TS_ERR_CUDA;
        return false;
    }
    q->full_left = r.steps / K;
    q->rem_left = r.steps % K;
    return true;
}

void ts_server::retire(Epoch &e, bool ok)
{
    const int64_t t = now_ns();
    const bool kernel_fault = e.err_copy != nullptr && *(volatile int *)e.err_copy != 0;
    for (auto &q : e.members) --q->inflight;
    for (auto &q : e.finishing) {
        if (q->state != R_ACTIVE) continue;
        if (!ok || kernel_fault) {
            q->state = R_FAILED;
            q->status = kernel_fault ? TS_ERR_TIMEOUT : TS_ERR_CUDA;
            snprintf(q->why, sizeof(q->why), "%s", kernel_fault ? "a bounded wait in the kernel gave up"
                                                                : "the epoch's event reported an error");
            ++failed;
        } else {
            q->state = R_DONE;
            q->status = TS_OK;
            q->t_done = t;
            ++completed;
            lat_ms.push_back((t - q->t_submit) * 1e-6);
            site_steps_done += (double)q->r.nx * q->r.ny * q->r.steps;
            t_last = t;
        }
    }
    if (kernel_fault) {
        // every request in this epoch shared the launch that reported it
        for (auto &q : e.members)
            if (q->state == R_ACTIVE) {
                q->state = R_FAILED;
                q->status = TS_ERR_TIMEOUT;
                ++failed;
            }
        cudaMemsetAsync(err_dev, 0, sizeof(int), compute);
    }
    active.erase(std::remove_if(active.begin(), active.end(),
                                [](const ReqP &q) { return q->state != R_ACTIVE; }),
                 active.end());
    cudaEventDestroy(e.done);
    cv_done.notify_all();
}

// Build and enqueue one epoch over the runnable grids (called with the lock
// held; releases it around CUDA calls that may block).
void ts_server::enqueue_epoch(std::unique_lock<std::mutex> &lk)
{
    ts::TraceRange trace_("server epoch");
    std::vector<ReqP> run_full, run_rem;
    for (auto &q : active) {
        if (q->cancel) continue;
        if (!q->ready_seen) {
            if (cudaEventQuery(q->ready) != cudaSuccess) continue;
            q->ready_seen = true;
        }
        if (q->full_left > 0)
            run_full.push_back(q);
        else if (q->rem_left > 0)
            run_rem.push_back(q);
    }
    if (run_full.empty() && run_rem.empty()) return;
    Epoch ep;
    const char *where = nullptr;   // the failing call, if any
    int64_t L = L_max;
    for (auto &q : run_full) L = std::min(L, q->full_left);
    lk.unlock();
    cudaError_t e = cudaSuccess;
    auto upload = [&](const std::vector<ReqP> &set, int depth, ts::MultiPlan &plan) -> int {
        const int slot = take_table();
        ts::EpochEntry *h = tab_host + (size_t)slot * cfg.max_slots;
        std::vector<int> nx(set.size()), ny(set.size());
        for (size_t i = 0; i < set.size(); ++i) {
            h[i] = ts::EpochEntry{set[i]->g->desc_dev, 0, set[i]->g->cur, 0};
            nx[i] = (int)set[i]->r.nx;
            ny[i] = (int)set[i]->r.ny;
        }
        plan = ts::fused_multi_plan(depth, (int)set.size(), nx.data(), ny.data(), h);
        if (plan.warps < 1 && e == cudaSuccess) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tab_dev + (size_t)slot * cfg.max_slots, h,
                                sizeof(ts::EpochEntry) * set.size(), cudaMemcpyHostToDevice, compute);
        ep.tables.push_back(slot);
        return slot;
    };
    if (!run_full.empty()) {
        ts::MultiPlan plan{};
        const int slot = upload(run_full, K, plan);
        if (e != cudaSuccess) where = "epoch table upload";
        if (e == cudaSuccess) {
            e = launch_full(slot, (int)run_full.size(), plan, (int)L);
            if (e != cudaSuccess) where = L > 1 ? "epoch graph" : "epoch launch";
        }
    }
    // remainder launches (one per distinct depth r < K)
    std::vector<std::vector<ReqP>> by_rem(K);
    for (auto &q : run_rem) by_rem[q->rem_left].push_back(q);
    for (int r = 1; r < K && e == cudaSuccess; ++r) {
        if (by_rem[r].empty()) continue;
        ts::MultiPlan plan{};
        const int slot = upload(by_rem[r], r, plan);
        if (e == cudaSuccess) {
            e = ts::launch_fused_multi(r, tab_dev + (size_t)slot * cfg.max_slots,
                                       (int)by_rem[r].size(), plan, 0, err_dev, compute);
            if (e != cudaSuccess) where = "remainder launch";
        }
    }
    ep.err_copy = err_host + (epochs % kTables);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ep.err_copy, err_dev, sizeof(int), cudaMemcpyDeviceToHost, compute);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ep.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ep.done, compute);
    for (int s : ep.tables)
        if (e == cudaSuccess) e = cudaEventRecord(tab_free[s], compute);
    if (e != cudaSuccess && !where) where = "epoch events";
    lk.lock();
    ++epochs;
    for (auto &q : run_full) {
        q->full_left -= L;
        if (L & 1) q->g->cur ^= 1;
        ++q->inflight;
        ep.members.push_back(q);
        if (q->full_left == 0 && q->rem_left == 0) ep.finishing.push_back(q);
    }
    for (auto &q : run_rem) {
        q->rem_left = 0;
        q->g->cur ^= 1;
        ++q->inflight;
        ep.members.push_back(q);
        ep.finishing.push_back(q);
    }
    if (e != cudaSuccess) {
        dead = true;
        for (auto &q : active) {
            q->state = R_FAILED;
            q->status = TS_ERR_CUDA;
            note(*q, where, e);
        }
        ts::set_error(TS_ERR_CUDA, "server: %s", cudaGetErrorString(e));
        cv_done.notify_all();
        return;
    }
    inflight.push_back(std::move(ep));
}

void ts_server::run()
{
    cudaSetDevice(device);   // a new thread starts on device 0 otherwise
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        // retire finished epochs
        while (!inflight.empty()) {
            cudaError_t q = cudaEventQuery(inflight.front().done);
            if (q == cudaErrorNotReady) break;
            retire(inflight.front(), q == cudaSuccess);
            inflight.pop_front();
        }
        // drop cancelled active requests once none of their work is in flight
        {
            bool any = false;
            for (auto &q : active)
                if (q->cancel && q->state == R_ACTIVE && q->inflight == 0) {
                    q->state = R_CANCELLED;
                    q->status = TS_ERR_STATE;
                    any = true;
                }
            if (any) {
                active.erase(std::remove_if(active.begin(), active.end(),
                                            [](const ReqP &q) { return q->state != R_ACTIVE; }),
                             active.end());
                cv_done.notify_all();
            }
        }
        if (stop && inflight.empty()) break;
        // admit in arrival order while memory and slots allow
        std::vector<ReqP> admitted;
        while (!stop && !dead && !pending.empty() &&
               (int)(active.size() + admitted.size()) < cfg.max_slots &&
               used + pending.front()->bytes <= cfg.hbm_budget_bytes) {
            ReqP q = pending.front();
            pending.pop_front();
            if (q->cancel) continue;
            used += q->bytes;
            q->reserved = true;
            peak = std::max(peak, used);
            admitted.push_back(q);
        }
        if (!admitted.empty()) {
            lk.unlock();
            std::vector<bool> ok(admitted.size());
            for (size_t i = 0; i < admitted.size(); ++i) ok[i] = admit_one(admitted[i]);
            lk.lock();
            const int64_t t = now_ns();
            for (size_t i = 0; i < admitted.size(); ++i) {
                ReqP &q = admitted[i];
                q->t_admit = t;
                if (!ok[i]) {
                    q->state = R_FAILED;
                    ++failed;
                    cv_done.notify_all();
                    continue;
                }
                if (q->r.steps == 0) {      // nothing to evolve
                    cudaEventSynchronize(q->ready);
                    q->state = R_DONE;
                    q->t_done = now_ns();
                    ++completed;
                    lat_ms.push_back((q->t_done - q->t_submit) * 1e-6);
                    cv_done.notify_all();
                    continue;
                }
                q->state = R_ACTIVE;
                active.push_back(q);
            }
        }
        // keep up to two epochs queued on the GPU
        if (!dead && inflight.size() < 2) {
            const size_t before = inflight.size();
            enqueue_epoch(lk);
            if (inflight.size() > before) continue;
        }
        // nothing to enqueue now: wait for the oldest epoch or for new work
        if (!inflight.empty()) {
            cudaEvent_t ev = inflight.front().done;
            lk.unlock();
            cudaEventSynchronize(ev);
            lk.lock();
        } else {
            cv_work.wait_for(lk, std::chrono::microseconds(200));
        }
    }
}

extern "C" {

ts_status ts_server_create(const ts_server_cfg *cfg, ts_server **out)
{
    if (!cfg || !out) return err(TS_ERR_ARG, "ts_server_create: null argument");
    if (cfg->max_slots < 1 || cfg->max_slots > 4096 || cfg->K < 0 || cfg->K > ts::FUSED_MAX_K ||
        cfg->hbm_budget_bytes == 0)
        return err(TS_ERR_ARG, "ts_server_create: need 1 <= max_slots <= 4096, 0 <= K <= 8, a budget");
    ts_server *s = new (std::nothrow) ts_server();
    if (!s) return err(TS_ERR_OOM, "ts_server_create: host allocation failed");
    s->cfg = *cfg;
    s->K = cfg->K == 0 ? 4 : cfg->K;
    cudaGetDevice(&s->device);
    const int steps_per_epoch = cfg->max_epoch_steps > 0 ? cfg->max_epoch_steps : 32;
    s->L_max = std::max(1, steps_per_epoch / s->K);
    cudaError_t e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaHostAlloc((void **)&s->err_host, sizeof(int) * kTables, cudaHostAllocDefault);
    if (e == cudaSuccess) {
        std::memset(s->err_host, 0, sizeof(int) * kTables);
        e = cudaMalloc((void **)&s->err_dev, sizeof(int));
    }
    if (e == cudaSuccess) e = cudaMemset(s->err_dev, 0, sizeof(int));
    // kernel attributes and occupancy are set up here, outside any capture
    for (int k = 1; k <= s->K && e == cudaSuccess; ++k) e = ts::fused_multi_prepare(k);
    const size_t tab_bytes = sizeof(ts::EpochEntry) * (size_t)kTables * cfg->max_slots;
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->tab_dev, tab_bytes);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->tab_host, tab_bytes, cudaHostAllocDefault);
    for (int i = 0; i < kTables && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&s->tab_free[i], cudaEventDisableTiming);
    if (e == cudaSuccess) {
        // keep freed request slabs in the pool for reuse
        int dev = 0;
        cudaGetDevice(&dev);
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (e != cudaSuccess) {
        ts_server_destroy(s);
        return err(TS_ERR_CUDA, "ts_server_create: %s", cudaGetErrorString(e));
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return TS_OK;
}

ts_status ts_server_submit(ts_server *s, const ts_request *r, uint64_t *ticket)
{
    if (!s || !r || !ticket) return err(TS_ERR_ARG, "ts_server_submit: null argument");
    if (!r->psi_re || !r->psi_im) return err(TS_ERR_ARG, "ts_server_submit: initial state missing");
    if (r->steps < 0) return err(TS_ERR_ARG, "ts_server_submit: negative step count");
    if (r->where != TS_HOST && r->where != TS_DEVICE)
        return err(TS_ERR_ARG, "ts_server_submit: unknown memory kind");
    if (r->psi_dtype != TS_F32 && r->psi_dtype != TS_F64)
        return err(TS_ERR_ARG, "ts_server_submit: unknown dtype");
    if (!std::isfinite(r->dt) || !std::isfinite(r->theta) || std::fabs(r->theta) > 0.25 * M_PI)
        return err(TS_ERR_ARG, "ts_server_submit: need finite dt and |theta| <= pi/4");
    ts_layout L;
    ts_status st = ts_grid_layout(r->nx, r->ny, TS_F32, &L);
    if (st != TS_OK) return st;
    auto q = std::make_shared<Req>();
    q->r = *r;
    q->bytes = L.slab_bytes;
    q->t_submit = now_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->dead) return err(TS_ERR_CUDA, "ts_server_submit: the server stopped after a CUDA error");
    if (q->bytes > s->cfg.hbm_budget_bytes)
        return err(TS_ERR_BUSY, "ts_server_submit: %lld x %lld needs %zu bytes, the budget is %zu",
                   (long long)r->nx, (long long)r->ny, q->bytes, s->cfg.hbm_budget_bytes);
    q->ticket = s->next_ticket++;
    s->reqs[q->ticket] = q;
    s->pending.push_back(q);
    ++s->submitted;
    if (s->t_first == 0) s->t_first = q->t_submit;
    *ticket = q->ticket;
    s->cv_work.notify_one();
    return TS_OK;
}

static void fill_result(const Req &q, ts_result *out)
{
    if (!out) return;
    out->status = q.state == R_DONE ? TS_OK
                  : (q.state == R_PENDING || q.state == R_ACTIVE) ? 1
                                                                  : (int)q.status;
    out->latency_ns = q.t_done ? q.t_done - q.t_submit : 0;
    out->queue_ns = q.t_admit ? q.t_admit - q.t_submit : 0;
    out->nx = q.r.nx;
    out->ny = q.r.ny;
    out->steps = q.r.steps;
}

ts_status ts_server_poll(ts_server *s, uint64_t ticket, ts_result *out)
{
    if (!s) return err(TS_ERR_ARG, "ts_server_poll: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return err(TS_ERR_ARG, "ts_server_poll: unknown ticket");
    fill_result(*it->second, out);
    return TS_OK;
}

ts_status ts_server_wait(ts_server *s, uint64_t ticket, int64_t timeout_ms, ts_result *out)
{
    if (!s) return err(TS_ERR_ARG, "ts_server_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return err(TS_ERR_ARG, "ts_server_wait: unknown ticket");
    ReqP q = it->second;
    auto finished = [&] { return q->state != R_PENDING && q->state != R_ACTIVE; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, finished);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) {
        fill_result(*q, out);
        return err(TS_ERR_TIMEOUT, "ts_server_wait: ticket %llu not done after %lld ms",
                   (unsigned long long)ticket, (long long)timeout_ms);
    }
    fill_result(*q, out);
    if (q->state == R_CANCELLED) return err(q->status, "ts_server_wait: request cancelled");
    if (q->state != R_DONE) return err(q->status, "ts_server_wait: request failed (%s)", q->why);
    return TS_OK;
}

ts_status ts_server_fetch(ts_server *s, uint64_t ticket, void *re, void *im, ts_dtype dtype,
                          ts_mem where)
{
    if (!s || !re || !im) return err(TS_ERR_ARG, "ts_server_fetch: null argument");
    ReqP q;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return err(TS_ERR_ARG, "ts_server_fetch: unknown ticket");
        q = it->second;
        if (q->state != R_DONE) return err(TS_ERR_STATE, "ts_server_fetch: request not done");
    }
    return ts_get_state(q->g, re, im, dtype, where, s->copy);
}

static void free_request(ts_server *s, Req &q)
{
    if (q.g) {
        ts_destroy_grid(q.g);   // does not free a caller-provided slab
        q.g = nullptr;
    }
    if (q.slab) {
        cudaFreeAsync(q.slab, s->copy);
        q.slab = nullptr;
    }
    if (q.ready) {
        cudaEventDestroy(q.ready);
        q.ready = nullptr;
    }
}

ts_status ts_server_release(ts_server *s, uint64_t ticket)
{
    if (!s) return err(TS_ERR_ARG, "ts_server_release: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return err(TS_ERR_ARG, "ts_server_release: unknown ticket");
    ReqP q = it->second;
    if (q->state == R_PENDING || q->state == R_ACTIVE)
        return err(TS_ERR_STATE, "ts_server_release: request still running (cancel it first)");
    free_request(s, *q);
    if (q->reserved) {
        s->used -= q->bytes;
        q->reserved = false;
    }
    s->reqs.erase(it);
    s->cv_work.notify_one();
    return TS_OK;
}

ts_status ts_server_cancel(ts_server *s, uint64_t ticket)
{
    if (!s) return err(TS_ERR_ARG, "ts_server_cancel: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return err(TS_ERR_ARG, "ts_server_cancel: unknown ticket");
    ReqP q = it->second;
    if (q->state == R_PENDING) {
        q->cancel = true;
        q->state = R_CANCELLED;
        q->status = TS_ERR_STATE;
        s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), q), s->pending.end());
        s->cv_done.notify_all();
    } else if (q->state == R_ACTIVE) {
        q->cancel = true;   // leaves at the next epoch boundary
    }
    return TS_OK;
}

ts_status ts_server_stats(ts_server *s, ts_server_metrics *out)
{
    if (!s || !out) return err(TS_ERR_ARG, "ts_server_stats: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->active = (int64_t)s->active.size();
    out->pending = (int64_t)s->pending.size();
    out->bytes_in_use = s->used;
    out->peak_bytes = s->peak;
    out->epochs = s->epochs;
    out->graph_launches = s->graph_launches;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const double pos = p * (double)(v.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - (double)i;
            return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
    }
    if (s->t_last > s->t_first)
        out->site_steps_per_s = s->site_steps_done / ((s->t_last - s->t_first) * 1e-9);
    return TS_OK;
}

ts_status ts_server_destroy(ts_server *s)
{
    if (!s) return TS_OK;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            for (auto &q : s->active) q->cancel = true;
            for (auto &q : s->pending) {
                q->state = R_CANCELLED;
                q->status = TS_ERR_STATE;
            }
            s->pending.clear();
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (auto &kv : s->reqs) free_request(s, *kv.second);
    s->reqs.clear();
    for (auto &kv : s->graphs) cudaGraphExecDestroy(kv.second);
    for (int i = 0; i < kTables; ++i)
        if (s->tab_free[i]) cudaEventDestroy(s->tab_free[i]);
    if (s->copy) cudaStreamSynchronize(s->copy);
    if (s->tab_dev) cudaFree(s->tab_dev);
    if (s->tab_host) cudaFreeHost(s->tab_host);
    if (s->err_host) cudaFreeHost(s->err_host);
    if (s->err_dev) cudaFree(s->err_dev);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    delete s;
    return TS_OK;
}

}  // extern "C"
