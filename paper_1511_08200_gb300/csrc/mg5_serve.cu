// mg5_serve.cu -- continuous-batching solve server (host runtime, C ABI in mg5.h).
//
// `slots` worker threads each own a non-blocking CUDA stream and a context
// (for the solves that run host-driven).  Requests queue in arrival order and
// a free worker takes the oldest.  Solves run as captured CUDA graphs from a
// pool shared by all workers (MG5_MIXED always; MG5_FP64 when the V-cycle can
// be captured: two grids or more, nu1 + nu2 even): a worker checks out an idle
// entry for the request's (grid size, parameters, gradient), replays it on
// its own stream and returns it, so a capture is paid once per key and per
// concurrent use, not per worker.  Up to `slots` solves are on the GPU at
// once, overlapping on the workers' streams.
//
// Memory: the server budget covers the pool's entries, the workers' own
// hierarchies and entries being built.  A request that does not fit evicts
// idle pool entries (least recently used first) and asks idle workers to drop
// their cached hierarchies; otherwise it waits for running solves to
// return theirs.  A request larger than the whole budget is refused at submit.
//
// A key holds at most kDupCap entries: when they are all busy, the request runs
// host-driven on the worker's own context (for mixed solves as fast as a replay
// under concurrency, measured) instead of building another, since building allocates and instantiates, which stalls the
// solves in flight.  Captures and device frees are serialised by one gate that
// host-driven solves hold shared: a free or a device-wide synchronisation in another
// thread can end a capture in progress.  A capture that fails anyway is retried once, then the
// request runs host-driven on the worker's own context.  Every solve is
// deterministic (fixed-order reductions, nothing shared between solves in
// flight), so a result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <thread>
#include <vector>

#include "mg5.h"
#include "mg5_mixed.cuh"
#include "mg5_pool.h"

namespace {

constexpr int kDupCap = 2;   // pooled graphs per (grid size, parameters, gradient)

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    mg5_request req;
    double t_submit;
};

// The footprint a request needs on a server that holds nothing.
int request_bytes(const mg5_request &r, size_t *need)
{
    const int rc = mg5_workspace_bytes(r.N, r.params.precision, need);   // checks N
    if (rc == MG5_OK && mg5::graph_capturable(r.N, &r.params))
        *need = mg5::graph_bytes(r.N, r.params.precision, r.grad != nullptr);
    return rc;
}

}  // namespace

struct mg5_server {
    int device = 0;
    size_t budget = 0;
    std::mutex mu;                     // queue, completions, byte counts, the pool's list
    std::condition_variable cv_work;   // queue changed / memory freed / stopping
    std::condition_variable cv_done;   // a completion arrived
    std::deque<Job> queue;
    std::deque<mg5_completion> done;
    std::vector<std::thread> workers;
    std::vector<size_t> held;          // bytes of each worker's own context
    mg5_ctx *pool = nullptr;           // graph entries shared by the workers
    size_t reserved = 0;               // bytes of entries being built
    std::shared_mutex gate;            // exclusive: capture, free; shared: host-driven solves
    int running = 0;
    bool stop = false;
    bool pressure = false;             // a worker waits for memory
    double t0 = 0.0;
    mg5_server_stats stats{};

    size_t total_locked() const
    {
        size_t t = reserved + mg5::graph_held(pool);
        for (size_t b : held)
            t += b;
        return t;
    }
};

namespace {

// Drop this worker's cached FP64 hierarchies (called with srv->mu held; returns with it held).
void release_own(mg5_server *srv, int w, mg5_ctx *ctx, std::unique_lock<std::mutex> &lk)
{
    lk.unlock();
    {
        std::unique_lock<std::shared_mutex> g(srv->gate);
        mg5_release(ctx);
    }
    lk.lock();
    srv->held[w] = mg5_bytes_held(ctx);
    srv->cv_work.notify_all();
}

// Free one idle pool entry (srv->mu held on entry and exit); false if none is idle.
bool evict_one(mg5_server *srv, std::unique_lock<std::mutex> &lk)
{
    GraphEntry *v = mg5::graph_take_idle(srv->pool);
    if (!v)
        return false;
    srv->stats.evictions++;
    lk.unlock();
    {
        std::unique_lock<std::shared_mutex> g(srv->gate);
        mg5::graph_free(v);
    }
    lk.lock();
    srv->cv_work.notify_all();
    return true;
}

// Wait for `need` more bytes (srv->mu held).  Returns false when nothing can
// free enough: nothing runs and nothing else is held or being built.
bool wait_for_bytes(mg5_server *srv, int w, mg5_ctx *ctx, size_t need,
                    std::unique_lock<std::mutex> &lk)
{
    for (;;) {
        if (!srv->budget || srv->total_locked() + need <= srv->budget)
            return true;
        if (evict_one(srv, lk))
            continue;
        if (srv->held[w] > 0 && ctx) {
            release_own(srv, w, ctx, lk);
            continue;
        }
        if (srv->running == 1 && srv->total_locked() == 0)
            return false;   // only this request, and it cannot fit
        srv->pressure = true;
        srv->cv_work.notify_all();
        srv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
    }
}

int run_on_worker(mg5_server *srv, int w, mg5_ctx *ctx, cudaStream_t st, const mg5_request &r,
             mg5_completion *c);

int run_pooled(mg5_server *srv, int w, mg5_ctx *ctx, cudaStream_t st, cudaEvent_t ev,
               const mg5_request &r, mg5_completion *c)
{
    const bool grad = r.grad != nullptr;
    GraphEntry *g = nullptr;
    size_t need = 0;
    bool host_driven = false;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        for (;;) {
            if ((g = mg5::graph_checkout(srv->pool, r.N, &r.params, grad)))
                break;
            if (mg5::graph_count(srv->pool, r.N, &r.params, grad) >= kDupCap) {
                host_driven = true;   // every entry of this key is busy
                break;
            }
            need = mg5::graph_bytes(r.N, r.params.precision, grad);
            if (!srv->budget || srv->total_locked() + need <= srv->budget) {
                srv->reserved += need;   // built below, outside the lock
                break;
            }
            // no idle entry of this key and no room for one: free something, or wait
            if (evict_one(srv, lk))
                continue;
            if (srv->held[w] > 0 && ctx) {
                release_own(srv, w, ctx, lk);
                continue;
            }
            if (srv->running == 1 && srv->total_locked() == 0)
                return MG5_E_OOM;
            srv->stats.memory_waits++;
            srv->pressure = true;
            srv->cv_work.notify_all();
            srv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
        }
        srv->pressure = false;
    }
    if (host_driven)
        return run_on_worker(srv, w, ctx, st, r, c);   // the worker-context path (any precision)
    c->t_admit = now_s() - srv->t0;
    if (!g) {
        std::string err;
        int rc = MG5_E_CUDA;
        const double tb = now_s();
        for (int attempt = 0; attempt < 2 && rc != MG5_OK && rc != MG5_E_OOM; ++attempt) {
            std::unique_lock<std::shared_mutex> gl(srv->gate);
            rc = mg5::graph_build_in(srv->pool, r.N, &r.params, grad, &g, &err);
        }
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->reserved -= need;
            srv->stats.builds++;
            srv->stats.build_seconds += now_s() - tb;
            if (rc == MG5_OK)
                mg5::graph_insert(srv->pool, g);
            else
                srv->stats.fallbacks++;
        }
        srv->cv_work.notify_all();
        if (rc != MG5_OK) {
            // no graph: the same solve, host-driven, on the worker's own context
            std::shared_lock<std::shared_mutex> gl(srv->gate);
            return mg5_solve_fifth_force(ctx, r.delta, r.N, &r.params, 0, r.phi, r.grad, &c->info,
                                         (void *)st);
        }
    }
    std::string err;
    int rc = mg5::graph_enqueue(g, r.delta, r.phi, r.grad, st, &err);
    if (rc == MG5_OK && mg5::host_wait(st, ev) != cudaSuccess) {
        cudaGetLastError();
        rc = MG5_E_CUDA;
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (rc == MG5_OK)
            rc = mg5::graph_finish(g, &c->info);
        else
            mg5::graph_checkin(g);
    }
    srv->cv_work.notify_all();
    return rc;
}

// A solve on the worker's own context, host-driven (requests that cannot be captured, and
// those whose pooled graphs are all busy): its hierarchy stays cached there.
int run_on_worker(mg5_server *srv, int w, mg5_ctx *ctx, cudaStream_t st, const mg5_request &r,
             mg5_completion *c)
{
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        size_t extra = 0;
        if (mg5_cached_bytes(ctx, r.N, r.params.precision, &extra) != MG5_OK)
            return MG5_E_ARG;
        if (extra && !wait_for_bytes(srv, w, ctx, extra, lk))
            return MG5_E_OOM;
        srv->held[w] += extra;   // reserve the footprint before the solve allocates it
        srv->pressure = false;
    }
    c->t_admit = now_s() - srv->t0;
    std::shared_lock<std::shared_mutex> gl(srv->gate);
    return mg5_solve_fifth_force(ctx, r.delta, r.N, &r.params, 0, r.phi, r.grad, &c->info,
                                 (void *)st);
}

void worker_main(mg5_server *srv, int w)
{
    cudaSetDevice(srv->device);
    mg5_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;   // the worker sleeps while its solve runs: many workers, few cores
    int rc_init = mg5_create(&ctx, srv->device, 0);
    if (rc_init == MG5_OK)
        rc_init = mg5_set_blocking_wait(ctx, 1);
    if (rc_init == MG5_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        rc_init = MG5_E_CUDA;
    if (rc_init == MG5_OK &&
        cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess)
        rc_init = MG5_E_CUDA;
    for (;;) {
        Job job;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                if (srv->stop && srv->queue.empty())
                    goto out;
                if (srv->pressure && srv->held[w] > 0 && ctx) {
                    release_own(srv, w, ctx, lk);   // a request waits for memory
                    continue;
                }
                if (!srv->queue.empty())
                    break;
                srv->cv_work.wait(lk);
            }
            job = srv->queue.front();
            srv->queue.pop_front();
            srv->running++;
        }
        mg5_completion c;
        std::memset(&c, 0, sizeof(c));
        c.tag = job.req.tag;
        c.t_submit = job.t_submit;
        if (rc_init != MG5_OK) {
            c.status = rc_init;
            c.t_admit = now_s() - srv->t0;
        } else if (mg5::graph_capturable(job.req.N, &job.req.params)) {
            c.status = run_pooled(srv, w, ctx, st, ev, job.req, &c);
        } else {
            c.status = run_on_worker(srv, w, ctx, st, job.req, &c);
        }
        if (c.status < 0 && c.info.status == 0)
            c.info.status = c.status;
        c.t_done = now_s() - srv->t0;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->held[w] = ctx ? mg5_bytes_held(ctx) : 0;
            srv->running--;
            srv->stats.completed++;
            srv->done.push_back(c);
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
out:
    if (ev)
        cudaEventDestroy(ev);
    if (st)
        cudaStreamDestroy(st);
    if (ctx) {
        std::unique_lock<std::shared_mutex> g(srv->gate);
        mg5_destroy(ctx);
    }
}

}  // namespace

extern "C" {

int mg5_server_create(mg5_server **out, int device, int slots, size_t hbm_budget_bytes)
{
    if (!out || slots < 1 || slots > 256)
        return MG5_E_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return MG5_E_CUDA;
    }
    if (device < 0 || device >= ndev)
        return MG5_E_ARG;
    mg5_ctx *pool = nullptr;
    if (int rc = mg5_create(&pool, device, 0))
        return rc;
    mg5_server *s = new mg5_server();
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->pool = pool;
    s->t0 = now_s();
    s->held.assign(slots, 0);
    for (int w = 0; w < slots; ++w)
        s->workers.emplace_back(worker_main, s, w);
    *out = s;
    return MG5_OK;
}

int mg5_server_submit(mg5_server *s, const mg5_request *req)
{
    if (!s || !req || !req->delta || !req->phi)
        return MG5_E_ARG;
    size_t need = 0;
    if (request_bytes(*req, &need) != MG5_OK)
        return MG5_E_ARG;
    if (s->budget && need > s->budget)
        return MG5_E_OOM;   // could never be admitted
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop)
            return MG5_E_ARG;
        s->queue.push_back(Job{*req, now_s() - s->t0});
    }
    s->cv_work.notify_all();
    return MG5_OK;
}

int mg5_server_poll(mg5_server *s, mg5_completion *out, int max, int wait_ms)
{
    if (!s || (!out && max > 0) || max < 0)
        return MG5_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    return n;
}

int mg5_server_pending(mg5_server *s, int *queued, int *running)
{
    if (!s)
        return MG5_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued)
        *queued = (int)s->queue.size();
    if (running)
        *running = s->running;
    return MG5_OK;
}

double mg5_server_clock(mg5_server *s) { return s ? now_s() - s->t0 : 0.0; }

size_t mg5_server_bytes_held(mg5_server *s)
{
    if (!s)
        return 0;
    std::lock_guard<std::mutex> lk(s->mu);
    return s->total_locked();
}

int mg5_server_get_stats(mg5_server *s, mg5_server_stats *out)
{
    if (!s || !out)
        return MG5_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return MG5_OK;
}

int mg5_server_destroy(mg5_server *s)
{
    if (!s)
        return MG5_E_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (std::thread &t : s->workers)
        t.join();
    mg5_destroy(s->pool);
    delete s;
    return MG5_OK;
}

}  // extern "C"
