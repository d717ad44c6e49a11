// mg5_serve.cu -- continuous-batching solve server (host runtime, C ABI in mg5.h).
//
// `slots` worker threads each own a context (its resident multigrid
// hierarchies, scalars and partial sums) and a non-blocking CUDA stream.
// Requests queue in arrival order.  A free worker admits the request at the
// head of the queue once the HBM footprint the request adds (a hierarchy for a
// grid size the worker has not cached yet) fits the server budget next to
// what every worker holds; if not, the worker first drops its own cached
// hierarchies, then waits for others to finish.  Admitted solves run
// concurrently on their workers' streams, so requests that arrive while
// others are on the GPU start as soon as a slot and memory free up.  Mixed
// solves run as cached CUDA graphs (mg5_solve_fifth_force with MG5_GRAPH).  Every
// solve is deterministic (fixed-order reductions, no state shared between
// workers), so a result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "mg5.h"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    mg5_request req;
    double t_submit;
};

// The footprint a request needs on a worker that holds nothing: the cached
// graph of a mixed solve, the hierarchy of an FP64 solve.
int request_bytes(const mg5_request &r, size_t *need)
{
    if (r.params.precision == MG5_MIXED)
        return mg5_graph_workspace_bytes(r.N, r.grad != nullptr, need);
    return mg5_workspace_bytes(r.N, r.params.precision, need);
}

}  // namespace

struct mg5_server {
    int device = 0;
    size_t budget = 0;
    std::mutex mu;
    std::condition_variable cv_work;   // queue changed / memory freed / stopping
    std::condition_variable cv_done;   // a completion arrived
    std::deque<Job> queue;
    std::deque<mg5_completion> done;
    std::vector<std::thread> workers;
    std::vector<size_t> held;          // bytes each worker's context holds
    int running = 0;
    bool stop = false;
    bool pressure = false;             // the queue head waits for memory
    double t0 = 0.0;
};

static void worker_main(mg5_server *srv, int w)
{
    cudaSetDevice(srv->device);
    mg5_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    int rc_init = mg5_create(&ctx, srv->device, 0);
    if (rc_init == MG5_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        rc_init = MG5_E_CUDA;
    auto release_own = [&](std::unique_lock<std::mutex> &lk) {
        lk.unlock();
        mg5_release(ctx);
        lk.lock();
        srv->held[w] = mg5_bytes_held(ctx);
        srv->cv_work.notify_all();
    };
    for (;;) {
        Job job;
        double t_admit = 0.0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                if (srv->stop && srv->queue.empty())
                    goto out;
                if (srv->pressure && srv->held[w] > 0 && ctx) {
                    release_own(lk);   // an admission is waiting for memory
                    continue;
                }
                if (srv->queue.empty()) {
                    srv->cv_work.wait(lk);
                    continue;
                }
                const mg5_request &r = srv->queue.front().req;
                size_t extra = 0;
                const int rcb = r.params.precision == MG5_MIXED
                                    ? mg5_graph_cached_bytes(ctx, r.N, &r.params, r.grad != nullptr, &extra)
                                    : mg5_cached_bytes(ctx, r.N, r.params.precision, &extra);
                if (rc_init == MG5_OK && srv->budget && rcb == MG5_OK) {
                    size_t total = 0;
                    for (size_t b : srv->held)
                        total += b;
                    if (total + extra > srv->budget) {
                        if (srv->held[w] > 0) {
                            release_own(lk);
                            continue;
                        }
                        if (srv->running == 0 && total == 0) {
                            // cannot fit on an empty server: complete it as out of memory
                            mg5_completion c;
                            std::memset(&c, 0, sizeof(c));
                            c.tag = srv->queue.front().req.tag;
                            c.t_submit = srv->queue.front().t_submit;
                            c.t_admit = c.t_done = now_s() - srv->t0;
                            c.status = MG5_E_OOM;
                            c.info.status = MG5_E_OOM;
                            srv->queue.pop_front();
                            srv->pressure = false;
                            srv->done.push_back(c);
                            srv->cv_done.notify_all();
                            continue;
                        }
                        srv->pressure = true;
                        srv->cv_work.notify_all();
                        srv->cv_work.wait(lk);
                        continue;
                    }
                }
                job = srv->queue.front();
                srv->queue.pop_front();
                srv->pressure = false;
                srv->running++;
                t_admit = now_s() - srv->t0;
                // reserve the footprint before the solve allocates it
                srv->held[w] += extra;
                break;
            }
        }
        mg5_completion c;
        std::memset(&c, 0, sizeof(c));
        c.tag = job.req.tag;
        c.t_submit = job.t_submit;
        c.t_admit = t_admit;
        if (rc_init != MG5_OK) {
            c.status = rc_init;
        } else {
            // mixed solves replay a cached CUDA graph (one launch, one synchronisation)
            const unsigned flags = job.req.params.precision == MG5_MIXED ? MG5_GRAPH : 0u;
            c.status = mg5_solve_fifth_force(ctx, job.req.delta, job.req.N, &job.req.params, flags,
                                             job.req.phi, job.req.grad, &c.info, (void *)st);
        }
        c.t_done = now_s() - srv->t0;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            srv->held[w] = ctx ? mg5_bytes_held(ctx) : 0;
            srv->running--;
            srv->done.push_back(c);
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
out:
    if (st)
        cudaStreamDestroy(st);
    if (ctx)
        mg5_destroy(ctx);
}

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
    mg5_server *s = new mg5_server();
    s->device = device;
    s->budget = hbm_budget_bytes;
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
    size_t t = 0;
    for (size_t b : s->held)
        t += b;
    return t;
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
    delete s;
    return MG5_OK;
}

}  // extern "C"
