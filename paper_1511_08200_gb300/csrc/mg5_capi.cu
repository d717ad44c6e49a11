// mg5_capi.cu -- host engine and C ABI of the mg5 library (see include/mg5.h).
//
// The context owns, per grid size, a resident multigrid hierarchy (device
// buffers), a partial-sum buffer for deterministic reductions and a block of
// per-grid device scalars (c, residual mean and norm).  The V-cycle schedule
// runs on the host and launches one kernel per step on the caller's stream;
// the only device->host traffic inside a solve is one 8-byte residual read
// per cycle (the convergence test of Sec. 3.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "mg5.h"
#include "mg5_kernels.cuh"
#include "mg5_mixed.cuh"
#include "mg5_pool.h"
#include "mg5_prof.cuh"

using namespace mg5;

namespace mg5 {
static std::atomic<long long> g_launches{0};
void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace mg5

namespace {

constexpr int kMaxLevels = 16;
constexpr int kMaxCoarsest = 32;
constexpr double kCoarseRtol = 1e-3;

struct Hier {
    int N = 0;
    int nlev = 0;
    int n[kMaxLevels] = {};
    double *v[kMaxLevels] = {};    // level iterate (level 0: caller's phi at run time)
    double *tmp[kMaxLevels] = {};  // ping-pong partner
    double *f[kMaxLevels] = {};    // right-hand side
    double *v0[kMaxLevels] = {};   // restricted iterate before the coarse solve
    double2 *spec[2] = {};         // coarsest-grid DFT work (coarsest side >= kSpectralMinSide)
    size_t bytes = 0;
};

// Dirichlet patch hierarchy: interior dims halve while all are even and the half is >= 4.
struct PatchHier {
    int p[3] = {};
    int nlev = 0;
    int q[kMaxLevels][3] = {};
    double *v[kMaxLevels] = {};    // boxes (level 0: caller's box at run time)
    double *tmp[kMaxLevels] = {};
    double *v0[kMaxLevels] = {};   // boxes, l >= 1
    double *f[kMaxLevels] = {};    // interior-indexed right-hand sides
    unsigned char *mk[kMaxLevels] = {};   // coarse masks (l >= 1) of masked relaxations, lazily
    size_t bytes = 0;
};

int patch_levels(const int p[3], int q[][3])
{
    int L = 0;
    int c[3] = {p[0], p[1], p[2]};
    for (;;) {
        q[L][0] = c[0];
        q[L][1] = c[1];
        q[L][2] = c[2];
        ++L;
        bool ok = L < kMaxLevels;
        for (int a = 0; a < 3; ++a)
            ok = ok && (c[a] % 2 == 0) && (c[a] / 2 >= 4);
        if (!ok)
            break;
        for (int a = 0; a < 3; ++a)
            c[a] /= 2;
    }
    return L;
}

size_t box_cells(const int q[3]) { return (size_t)(q[0] + 2) * (q[1] + 2) * (q[2] + 2); }
size_t int_cells(const int q[3]) { return (size_t)q[0] * q[1] * q[2]; }

int num_levels(int N, int *sizes)
{
    int L = 0, n = N;
    sizes[L++] = n;
    while ((n / 2) % 2 == 0 && n / 2 >= 4 && L < kMaxLevels) {
        n /= 2;
        sizes[L++] = n;
    }
    return L;
}

size_t fp64_bytes(int N)
{
    int sz[kMaxLevels];
    const int L = num_levels(N, sz);
    size_t b = 2 * (size_t)N * N * N * sizeof(double);  // tmp + f on the finest grid
    for (int l = 1; l < L; ++l)
        b += 4 * (size_t)sz[l] * sz[l] * sz[l] * sizeof(double);
    if (L > 1 && sz[L - 1] >= kSpectralMinSide)
        b += 2 * (size_t)sz[L - 1] * sz[L - 1] * sz[L - 1] * sizeof(double2);
    return b;
}

}  // namespace

// A captured batch: one graph with a branch per box (its own hierarchy,
// scalars and partial sums), each branch a WHILE loop of defect-correction
// steps whose condition a device kernel sets.
struct BatchSet {
    int nbox = 0;
    std::vector<int> N;
    std::vector<mg5_params> prm;
    std::vector<const double *> delta;
    std::vector<double *> phi, grad;
    std::vector<MixedHier *> hier;
    std::vector<double2 *> partials;
    std::vector<LevelScal *> ls;
    std::vector<SolveCounters *> cnt;
    BoxCtl *ctl = nullptr;
    std::vector<CaptureStats> stats;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t bytes = 0;
    unsigned long long sched = 0;   // schedule-table version at capture
};

// A mixed solve of one size and parameter set captured as a graph (defect-correction
// loop as a WHILE node), with its own hierarchy, scalars and staging buffers.
struct GraphReadback {
    BoxCtl ctl;
    SolveCounters cnt;
    LevelScal ls0;
    double c_in;   // patch form: the compatibility constant of this call (host -> device)
};

struct GraphEntry {
    int N = 0;
    mg5_params prm{};
    bool grad = false;
    bool fmg = false;              // FP64 form: full-multigrid start
    bool busy = false;
    MixedHier *hier = nullptr;     // MG5_MIXED
    Hier *hier64 = nullptr;        // MG5_FP64
    PatchHier *hierp = nullptr;    // Dirichlet patch relaxation (pf in pdims)
    int pdims[3] = {0, 0, 0};
    double *cdev = nullptr;        // patch form: device copy of the compatibility constant
    double2 *partials = nullptr;
    LevelScal *ls = nullptr;
    SolveCounters *cnt = nullptr;
    BoxCtl *ctl = nullptr;
    double *delta = nullptr, *phi = nullptr, *gout = nullptr;
    GraphReadback *rb = nullptr;   // pinned host copy of the control state
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CaptureStats stats{};
    size_t bytes = 0;              // device bytes, hierarchy included
    unsigned long long last_use = 0;
    unsigned long long sched = 0;  // schedule-table version at capture (see current())
    // replayable: the sweep schedules it was captured with are still the table's (patch
    // relaxations use no schedule)
    bool current() const { return hierp || sched == schedule_version(); }
};

constexpr size_t kGraphCacheMax = 48;   // entries per context on the single-caller path

struct mg5_ctx {
    int device = 0;
    size_t budget = 0;
    size_t held = 0;
    std::string err;
    std::vector<Hier *> hiers;
    std::vector<MixedHier *> mixed;
    std::vector<PatchHier *> patches;
    BatchSet *batch = nullptr;
    std::vector<GraphEntry *> graphs;
    unsigned long long graph_clock = 0;
    double2 *partials = nullptr;
    LevelScal *ls = nullptr;        // kScalSlots slots
    SolveCounters *cnt = nullptr;
    double *h_rel = nullptr;        // pinned host scalars
    // staging for MG5_HOST_IO and patch scratch
    double *stage = nullptr;
    size_t stage_bytes = 0;
    double *patch = nullptr;
    size_t patch_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t evb = nullptr;      // blocking-sync event: host waits sleep instead of spinning
    bool blocking = false;
    bool autotune = false;          // tune untuned grid sides before a solve
    Profiler prof;
};

// ------------------------------------------------------------ helpers

// A reduction's partial-sum buffer, zeroed: its last slot is the blocks-done counter of the
// reductions that finalize in their own last block (mg5_fin.cuh).
static cudaError_t alloc_partials(double2 **p)
{
    cudaError_t e = cudaMalloc((void **)p, sizeof(double2) * kMaxPartials);
    if (e == cudaSuccess)
        e = cudaMemset(*p, 0, sizeof(double2) * kMaxPartials);
    return e;
}

extern "C" {  // defined further down, inside the ABI block
static bool same_params(const mg5_params &a, const mg5_params &b);
static int solve_graph(mg5_ctx *ctx, const double *delta, int N, const mg5_params *p, double *phi,
                       double *grad, bool fmg, mg5_info *info, cudaStream_t st);
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return MG5_E_CUDA;                                                             \
        }                                                                                  \
    } while (0)

#define RET(x)                      \
    do {                            \
        int r_ = (x);               \
        if (r_ != MG5_OK)           \
            return r_;              \
    } while (0)

// Host wait for st on this context's solve paths (spin, or sleep when set to blocking).
static cudaError_t ctx_wait(mg5_ctx *ctx, cudaStream_t st)
{
    return host_wait(st, ctx->blocking ? ctx->evb : nullptr);
}

// Tune the sweep schedule of every non-coarsest grid side of N's hierarchy not in the table.
static int ctx_autotune(mg5_ctx *ctx, int N, int precision, cudaStream_t st)
{
    int sz[kMaxLevels];
    const int L = num_levels(N, sz);
    for (int l = 0; l + 1 < L; ++l) {
        if (sweep_tuned(ctx->device, precision, sz[l]))
            continue;
        const cudaError_t e = tune_side(ctx->device, precision, sz[l], st, nullptr);
        if (e != cudaSuccess) {
            ctx->err = std::string("autotune: ") + cudaGetErrorString(e);
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? MG5_E_OOM : MG5_E_CUDA;
        }
    }
    return MG5_OK;
}

static int ctx_alloc(mg5_ctx *ctx, void **p, size_t bytes)
{
    if (ctx->budget && ctx->held + bytes > ctx->budget) {
        ctx->err = "scratch would exceed the context's HBM budget";
        return MG5_E_OOM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? MG5_E_OOM : MG5_E_CUDA;
    }
    ctx->held += bytes;
    return MG5_OK;
}

static void ctx_free(mg5_ctx *ctx, void *p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        ctx->held -= bytes;
    }
}

static void free_hier(mg5_ctx *ctx, Hier *h)
{
    const size_t n3 = (size_t)h->N * h->N * h->N * sizeof(double);
    ctx_free(ctx, h->tmp[0], n3);
    ctx_free(ctx, h->f[0], n3);
    for (int l = 1; l < h->nlev; ++l) {
        const size_t b = (size_t)h->n[l] * h->n[l] * h->n[l] * sizeof(double);
        ctx_free(ctx, h->v[l], b);
        ctx_free(ctx, h->tmp[l], b);
        ctx_free(ctx, h->f[l], b);
        ctx_free(ctx, h->v0[l], b);
    }
    const int nc = h->n[h->nlev - 1];
    for (double2 *q : {h->spec[0], h->spec[1]})
        ctx_free(ctx, q, (size_t)nc * nc * nc * sizeof(double2));
    delete h;
}

// An FP64 hierarchy owned by a captured graph (plain allocations, counted by the entry).
static void free_hier_raw(Hier *h)
{
    if (!h)
        return;
    for (void *q : {(void *)h->tmp[0], (void *)h->f[0]})
        if (q)
            cudaFree(q);
    for (int l = 1; l < h->nlev; ++l)
        for (void *q : {(void *)h->v[l], (void *)h->tmp[l], (void *)h->f[l], (void *)h->v0[l]})
            if (q)
                cudaFree(q);
    for (void *q : {(void *)h->spec[0], (void *)h->spec[1]})
        if (q)
            cudaFree(q);
    delete h;
}

static cudaError_t alloc_hier_raw(int N, Hier **out)
{
    Hier *h = new Hier();
    h->N = N;
    h->nlev = num_levels(N, h->n);
    const size_t n3 = (size_t)N * N * N * sizeof(double);
    cudaError_t e = cudaMalloc((void **)&h->tmp[0], n3);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&h->f[0], n3);
    for (int l = 1; l < h->nlev && e == cudaSuccess; ++l) {
        const size_t b = (size_t)h->n[l] * h->n[l] * h->n[l] * sizeof(double);
        for (double **q : {&h->v[l], &h->tmp[l], &h->f[l], &h->v0[l]})
            if (e == cudaSuccess)
                e = cudaMalloc((void **)q, b);
    }
    const int nc = h->n[h->nlev - 1];
    if (e == cudaSuccess && h->nlev > 1 && nc >= kSpectralMinSide)
        for (double2 **q : {&h->spec[0], &h->spec[1]})
            if (e == cudaSuccess)
                e = cudaMalloc((void **)q, (size_t)nc * nc * nc * sizeof(double2));
    if (e != cudaSuccess) {
        free_hier_raw(h);
        return e;
    }
    h->bytes = fp64_bytes(N);
    *out = h;
    return cudaSuccess;
}

static int get_hier(mg5_ctx *ctx, int N, Hier **out)
{
    for (Hier *h : ctx->hiers)
        if (h->N == N) {
            *out = h;
            return MG5_OK;
        }
    Hier *h = new Hier();
    h->N = N;
    h->nlev = num_levels(N, h->n);
    int rc = MG5_OK;
    const size_t n3 = (size_t)N * N * N * sizeof(double);
    rc = ctx_alloc(ctx, (void **)&h->tmp[0], n3);
    if (rc == MG5_OK)
        rc = ctx_alloc(ctx, (void **)&h->f[0], n3);
    for (int l = 1; l < h->nlev && rc == MG5_OK; ++l) {
        const size_t b = (size_t)h->n[l] * h->n[l] * h->n[l] * sizeof(double);
        rc = ctx_alloc(ctx, (void **)&h->v[l], b);
        if (rc == MG5_OK)
            rc = ctx_alloc(ctx, (void **)&h->tmp[l], b);
        if (rc == MG5_OK)
            rc = ctx_alloc(ctx, (void **)&h->f[l], b);
        if (rc == MG5_OK)
            rc = ctx_alloc(ctx, (void **)&h->v0[l], b);
    }
    const int ncs = h->n[h->nlev - 1];
    if (rc == MG5_OK && h->nlev > 1 && ncs >= kSpectralMinSide)
        for (double2 **q : {&h->spec[0], &h->spec[1]})
            if (rc == MG5_OK)
                rc = ctx_alloc(ctx, (void **)q, (size_t)ncs * ncs * ncs * sizeof(double2));
    if (rc != MG5_OK) {
        free_hier(ctx, h);
        return rc;
    }
    h->bytes = fp64_bytes(N);
    ctx->hiers.push_back(h);
    *out = h;
    return MG5_OK;
}

static void free_patch(mg5_ctx *ctx, PatchHier *h)
{
    for (int l = 0; l < h->nlev; ++l) {
        const size_t bb = box_cells(h->q[l]) * sizeof(double), ib = int_cells(h->q[l]) * sizeof(double);
        if (l > 0) {
            ctx_free(ctx, h->v[l], bb);
            ctx_free(ctx, h->v0[l], bb);
        }
        ctx_free(ctx, h->tmp[l], bb);
        ctx_free(ctx, h->f[l], ib);
        if (h->mk[l])
            ctx_free(ctx, h->mk[l], int_cells(h->q[l]));
    }
    delete h;
}

// the coarse masks of a context-owned patch hierarchy (allocated on first use)
static int get_patch_masks(mg5_ctx *ctx, PatchHier *h)
{
    for (int l = 1; l < h->nlev; ++l)
        if (!h->mk[l]) {
            RET(ctx_alloc(ctx, (void **)&h->mk[l], int_cells(h->q[l])));
            h->bytes += int_cells(h->q[l]);
        }
    return MG5_OK;
}

// A patch hierarchy owned by a captured graph (plain allocations, counted by the entry).
static void free_patch_raw(PatchHier *h)
{
    if (!h)
        return;
    for (int l = 0; l < h->nlev; ++l)
        for (void *q : {(void *)h->v0[l], (void *)h->tmp[l], (void *)h->f[l],
                        l > 0 ? (void *)h->v[l] : nullptr})
            if (q)
                cudaFree(q);
    delete h;
}

static cudaError_t alloc_patch_raw(const int p[3], PatchHier **out)
{
    PatchHier *h = new PatchHier();
    for (int a = 0; a < 3; ++a)
        h->p[a] = p[a];
    h->nlev = patch_levels(p, h->q);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < h->nlev && e == cudaSuccess; ++l) {
        const size_t bb = box_cells(h->q[l]) * sizeof(double), ib = int_cells(h->q[l]) * sizeof(double);
        if (l > 0) {
            e = cudaMalloc((void **)&h->v[l], bb);
            if (e == cudaSuccess)
                e = cudaMalloc((void **)&h->v0[l], bb);
            h->bytes += 2 * bb;
        }
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&h->tmp[l], bb);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&h->f[l], ib);
        h->bytes += bb + ib;
    }
    if (e != cudaSuccess) {
        free_patch_raw(h);
        return e;
    }
    *out = h;
    return cudaSuccess;
}

static int get_patch(mg5_ctx *ctx, const int p[3], PatchHier **out)
{
    for (PatchHier *h : ctx->patches)
        if (h->p[0] == p[0] && h->p[1] == p[1] && h->p[2] == p[2]) {
            *out = h;
            return MG5_OK;
        }
    PatchHier *h = new PatchHier();
    for (int a = 0; a < 3; ++a)
        h->p[a] = p[a];
    h->nlev = patch_levels(p, h->q);
    int rc = MG5_OK;
    for (int l = 0; l < h->nlev && rc == MG5_OK; ++l) {
        const size_t bb = box_cells(h->q[l]) * sizeof(double), ib = int_cells(h->q[l]) * sizeof(double);
        if (l > 0) {
            rc = ctx_alloc(ctx, (void **)&h->v[l], bb);
            if (rc == MG5_OK)
                rc = ctx_alloc(ctx, (void **)&h->v0[l], bb);
            h->bytes += 2 * bb;
        }
        if (rc == MG5_OK)
            rc = ctx_alloc(ctx, (void **)&h->tmp[l], bb);
        if (rc == MG5_OK)
            rc = ctx_alloc(ctx, (void **)&h->f[l], ib);
        h->bytes += bb + ib;
    }
    if (rc != MG5_OK) {
        free_patch(ctx, h);
        return rc;
    }
    ctx->patches.push_back(h);
    *out = h;
    return MG5_OK;
}

static void free_batch(mg5_ctx *ctx)
{
    BatchSet *b = ctx->batch;
    if (!b)
        return;
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    if (b->graph)
        cudaGraphDestroy(b->graph);
    for (MixedHier *m : b->hier)
        free_mixed(m, &ctx->held);
    for (double2 *p : b->partials)
        if (p)
            cudaFree(p);
    for (LevelScal *p : b->ls)
        if (p)
            cudaFree(p);
    for (SolveCounters *p : b->cnt)
        if (p)
            cudaFree(p);
    if (b->ctl)
        cudaFree(b->ctl);
    ctx->held -= b->bytes;
    delete b;
    ctx->batch = nullptr;
}

static size_t graph_entry_bytes64(int N, bool grad)
{
    const size_t n3 = (size_t)N * N * N;
    return fp64_bytes(N) + n3 * sizeof(double) * (grad ? 5 : 2) + sizeof(double2) * kMaxPartials +
           sizeof(LevelScal) * kScalSlots + sizeof(SolveCounters) + sizeof(BoxCtl);
}

static size_t graph_entry_bytes(int N, bool grad)
{
    const size_t n3 = (size_t)N * N * N;
    return mixed_bytes(N) + n3 * sizeof(double) * (grad ? 5 : 2) + sizeof(double2) * kMaxPartials +
           sizeof(LevelScal) * kScalSlots + sizeof(SolveCounters) + sizeof(BoxCtl);
}

static int ensure_buffer(mg5_ctx *ctx, double **buf, size_t *have, size_t need)
{
    if (*have >= need)
        return MG5_OK;
    ctx_free(ctx, *buf, *have);
    *buf = nullptr;
    *have = 0;
    RET(ctx_alloc(ctx, (void **)buf, need));
    *have = need;
    return MG5_OK;
}

static int check_size(int N)
{
    if (N < 4 || (N & 1))
        return MG5_E_ARG;
    int sz[kMaxLevels];
    const int L = num_levels(N, sz);
    if (sz[L - 1] > kMaxCoarsest)
        return MG5_E_ARG;
    return MG5_OK;
}

static int check_params(const mg5_params *p)
{
    if (!p || !(p->h > 0.0) || !(p->alpha >= 0.0) || !std::isfinite(p->s) || !(p->tol >= 0.0) ||
        p->nu1 < 0 || p->nu2 < 0 || p->nu_coarse < 0 || p->max_cycles < 0 ||
        (p->precision != MG5_FP64 && p->precision != MG5_MIXED) || !(p->omega >= 0.0) ||
        !(p->omega < 2.0))
        return MG5_E_ARG;
    return MG5_OK;
}

// ------------------------------------------------------------ FP64 V-cycle engine

namespace {

struct Run64 {
    mg5_ctx *ctx;
    Hier *h;
    const mg5_params *p;
    cudaStream_t st;
    double hl[kMaxLevels];  // cell size per level
    long long cu = 0;       // cell updates of the non-coarsest sweeps
    // device scratch: the context's, or a captured graph's own
    LevelScal *lsb = nullptr;
    SolveCounters *cntb = nullptr;
    double2 *partb = nullptr;

    void bind_ctx_scratch()
    {
        lsb = ctx->ls;
        cntb = ctx->cnt;
        partb = ctx->partials;
    }
    bool bound() const { return lsb && cntb && partb; }
    LevelScal *ls(int l) { return lsb + l; }
    double *c(int l) { return &lsb[l].c; }
    double *m(int l) { return &lsb[l].m; }

    int sweep(int l)
    {
        const CoefT<double> cf = make_coef<double>(hl[l], p->alpha, omega_of(p));
        ProfScope ps(&ctx->prof, l == 0 ? PK_SWEEP64 : PK_SWEEP64C, st, (double)(h->n[l]) * (h->n[l]) * (h->n[l]));
        cudaError_t e = launch_sweep_sched<double>(sweep_schedule(ctx->device, MG5_FP64, h->n[l]),
                                                   h->v[l], h->tmp[l], h->f[l], c(l), h->n[l], cf,
                                                   &cntb->clamped, st);
        if (e != cudaSuccess) {
            ctx->err = std::string("sweep: ") + cudaGetErrorString(e);
            return MG5_E_CUDA;
        }
        std::swap(h->v[l], h->tmp[l]);
        cu += (long long)h->n[l] * h->n[l] * h->n[l];
        return MG5_OK;
    }

    // residual of level l, restricted onto l+1; finalize updates c_l and the norm
    int resid_restrict(int l)
    {
        const CoefT<double> cf = make_coef<double>(hl[l], p->alpha);
        int nb = 0;
        mg5_ctx *ctx = this->ctx;
        {
            ProfScope ps(&ctx->prof, PK_RESTRICT64, st, (double)(h->n[l]) * (h->n[l]) * (h->n[l]));
            const double n3 = (double)h->n[l] * h->n[l] * h->n[l];
            CK(launch_resid_restrict<double>(h->v[l], h->f[l], c(l), h->n[l], cf, h->v[l + 1],
                                             h->v0[l + 1], h->f[l + 1], partb, &nb, st, nullptr,
                                             Fin{ls(l), FIN_RESID, n3}));
        }
        return MG5_OK;
    }

    int residual_only(int l)
    {
        const CoefT<double> cf = make_coef<double>(hl[l], p->alpha);
        int nb = 0;
        mg5_ctx *ctx = this->ctx;
        const double n3 = (double)h->n[l] * h->n[l] * h->n[l];
        CK(launch_residual<double>(h->v[l], h->f[l], c(l), h->n[l], cf, nullptr, partb,
                                   &nb, st, Fin{ls(l), FIN_RESID, n3}));
        return MG5_OK;
    }

    int coarsest(int l)
    {
        const CoefT<double> cf = make_coef<double>(hl[l], p->alpha, omega_of(p));
        mg5_ctx *ctx = this->ctx;
        ProfScope ps(&ctx->prof, PK_COARSEST64, st);
        if (h->spec[0] && h->n[l] >= kSpectralMinSide) {
            CK(launch_coarsest_spectral<double>(h->v[l], h->tmp[l], h->f[l], h->n[l], cf, ls(l),
                                                kSpectralIters, &cntb->clamped, &cntb->coarse_sweeps,
                                                partb, h->spec[0], h->spec[1], st));
            return MG5_OK;
        }
        CK(launch_coarsest<double>(h->v[l], h->tmp[l], h->f[l], h->n[l], cf, c(l), p->nu_coarse,
                                   kCoarseRtol, &cntb->clamped, &cntb->coarse_sweeps, st));
        return MG5_OK;
    }

    // coarse-grid correction for level l-1, entered with v[l] = v0[l] = R v[l-1]
    // and f[l] = R r[l-1]
    int coarse_visit(int l)
    {
        mg5_ctx *ctx = this->ctx;
        const CoefT<double> cfc = make_coef<double>(hl[l], p->alpha);
        {
            ProfScope ps(&ctx->prof, PK_COARSE_RHS64, st, (double)(h->n[l]) * (h->n[l]) * (h->n[l]));
            CK(launch_coarse_rhs<double>(h->v[l], h->f[l], m(l - 1), c(l), h->n[l], cfc, st));
        }
        if (l == h->nlev - 1)
            return coarsest(l);
        for (int s = 0; s < p->nu1; ++s)
            RET(sweep(l));
        RET(resid_restrict(l));
        RET(coarse_visit(l + 1));
        {
            ProfScope ps(&ctx->prof, PK_PROLONG64, st, (double)(h->n[l]) * (h->n[l]) * (h->n[l]));
            CK(launch_prolong_add<double>(h->v[l + 1], h->v0[l + 1], h->n[l + 1], h->v[l], c(l),
                                          c(l + 1), st));
        }
        for (int s = 0; s < p->nu2; ++s)
            RET(sweep(l));
        return MG5_OK;
    }

    // one V-cycle with grid l as the finest grid (its f holds that grid's own rhs)
    int vcycle_top(int l)
    {
        mg5_ctx *ctx = this->ctx;
        for (int s = 0; s < p->nu1; ++s)
            RET(sweep(l));
        RET(resid_restrict(l));
        RET(coarse_visit(l + 1));
        CK(launch_prolong_add<double>(h->v[l + 1], h->v0[l + 1], h->n[l + 1], h->v[l], c(l),
                                      c(l + 1), st));
        for (int s = 0; s < p->nu2; ++s)
            RET(sweep(l));
        return MG5_OK;
    }

    // Full-multigrid start: the rhs restricted down the hierarchy, the coarsest
    // problem solved, then on each finer grid the interpolated coarse solution
    // (and c) improved by one V-cycle; the finest grid receives the interpolant.
    int fmg()
    {
        mg5_ctx *ctx = this->ctx;
        const int L = h->nlev;
        for (int l = 1; l < L; ++l)
            CK(launch_restrict<double>(h->f[l - 1], h->n[l - 1], h->f[l], st));
        const size_t nL = (size_t)h->n[L - 1] * h->n[L - 1] * h->n[L - 1];
        CK(cudaMemsetAsync(h->v[L - 1], 0, nL * sizeof(double), st));
        RET(coarsest(L - 1));
        for (int l = L - 2; l >= 0; --l) {
            const size_t nl = (size_t)h->n[l] * h->n[l] * h->n[l];
            CK(cudaMemsetAsync(h->v[l], 0, nl * sizeof(double), st));
            CK(cudaMemsetAsync(c(l), 0, sizeof(double), st));
            CK(launch_prolong_add<double>(h->v[l + 1], nullptr, h->n[l + 1], h->v[l], c(l), c(l + 1),
                                          st));
            if (l > 0)
                RET(vcycle_top(l));
        }
        return MG5_OK;
    }
};

}  // namespace

// Plain FP64 solve on device buffers.  phi holds the initial guess.
static int solve64(mg5_ctx *ctx, const double *delta, int N, const mg5_params *p, double *phi,
                   bool warm, bool fmg, mg5_info *info, cudaStream_t st)
{
    Hier *h = nullptr;
    RET(get_hier(ctx, N, &h));
    Run64 R{ctx, h, p, st, {}, 0};
    R.bind_ctx_scratch();
    if (!R.bound()) {
        ctx->err = "solve64: context scratch not allocated";
        return MG5_E_ARG;
    }
    for (int l = 0; l < h->nlev; ++l)
        R.hl[l] = p->h * (double)(1 << l);
    const long long n3 = (long long)N * N * N;
    CK(cudaMemsetAsync(ctx->ls, 0, sizeof(LevelScal) * kScalSlots, st));
    CK(cudaMemsetAsync(ctx->cnt, 0, sizeof(SolveCounters), st));
    int nb = 0;
    CK(launch_scale(delta, p->s, h->f[0], n3, ctx->partials, &nb, st, 0.0, nullptr,
                    Fin{ctx->ls, FIN_FNORM, (double)n3}));
    double *caller_phi = phi;
    h->v[0] = phi;
    // tmp[0] is the context's; v/tmp swap on every sweep.  Every exit path
    // hands tmp[0] back to the hierarchy.
    struct Restore {
        Hier *h;
        double *own;
        ~Restore()
        {
            h->v[0] = nullptr;
            h->tmp[0] = own;
        }
    } restore{h, h->tmp[0]};
    if (fmg && !warm && h->nlev > 1)
        RET(R.fmg());
    int status = MG5_E_NOT_CONVERGED;
    double best = INFINITY;
    int cyc = 0, nh = 0;    // nh: residual checks recorded (a warm start's check comes first)
    bool pre_check = warm;  // a warm start is tested (and c set) before any smoothing
    for (;; ++cyc) {
        if (pre_check) {
            RET(R.residual_only(0));
        } else if (h->nlev == 1) {
            RET(R.coarsest(0));
            RET(R.residual_only(0));
        } else {
            for (int s = 0; s < p->nu1; ++s)
                RET(R.sweep(0));
            RET(R.resid_restrict(0));
        }
        CK(cudaMemcpyAsync(ctx->h_rel, &ctx->ls[0].rel, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(ctx_wait(ctx, st));
        const double rel = *ctx->h_rel;
        if (info && nh < 64) {
            info->history[nh] = rel;
            info->n_history = nh + 1;
        }
        ++nh;
        if (info)
            info->rel_residual = rel;
        if (!std::isfinite(rel)) {
            status = MG5_E_NONFINITE;
            break;
        }
        if (rel <= p->tol) {
            status = MG5_OK;
            break;
        }
        best = std::min(best, rel);
        if (cyc >= 3 && rel > 10.0 * best) {
            status = MG5_E_DIVERGED;
            break;
        }
        if (pre_check) {
            pre_check = false;
            --cyc;   // the check of the initial guess is not a cycle
            continue;
        }
        if (cyc >= p->max_cycles) {
            status = MG5_E_NOT_CONVERGED;
            break;
        }
        if (h->nlev == 1)
            continue;
        RET(R.coarse_visit(1));
        {
            ProfScope ps(&ctx->prof, PK_PROLONG64, st, (double)(h->n[0]) * (h->n[0]) * (h->n[0]));
            CK(launch_prolong_add<double>(h->v[1], h->v0[1], h->n[1], h->v[0], R.c(0), R.c(1), st));
        }
        for (int s = 0; s < p->nu2; ++s)
            RET(R.sweep(0));
    }
    if (h->v[0] != caller_phi)
        CK(cudaMemcpyAsync(caller_phi, h->v[0], n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // gauge: subtract mean(phi)
    CK(launch_sum(caller_phi, n3, ctx->partials, &nb, st, Fin{ctx->ls, FIN_MEAN, (double)n3}));
    CK(launch_sub_mean(caller_phi, n3, &ctx->ls[0].mean, st));
    if (info) {
        info->cycles = cyc;
        info->levels = h->nlev;
        info->coarsest_n = h->n[h->nlev - 1];
        info->cell_updates = R.cu;   // coarsest sweeps are added by the caller
    }
    return status;
}

// ------------------------------------------------------------ C ABI

extern "C" {

int mg5_version(void) { return 100; }

long long mg5_kernel_launches(void) { return launches_total(); }

const char *mg5_status_string(int s)
{
    switch (s) {
    case MG5_OK: return "ok";
    case MG5_W_DISC_CLAMP: return "converged with clamped discriminants";
    case MG5_E_ARG: return "invalid argument";
    case MG5_E_OOM: return "out of memory (HBM budget)";
    case MG5_E_CUDA: return "CUDA error";
    case MG5_E_NOT_CONVERGED: return "not converged within max_cycles";
    case MG5_E_DIVERGED: return "diverged";
    case MG5_E_NONFINITE: return "non-finite residual";
    case MG5_E_TOO_LARGE: return "grid exceeds the entry point's fixed scratch";
    default: return "unknown status";
    }
}

int mg5_default_params(mg5_params *p)
{
    if (!p)
        return MG5_E_ARG;
    std::memset(p, 0, sizeof(*p));
    p->tol = 1e-10;
    p->nu1 = 2;
    p->nu2 = 2;
    p->nu_coarse = 500;
    p->max_cycles = 100;
    p->precision = MG5_FP64;
    return MG5_OK;
}

int mg5_ndgp_coefficients(double a, double omega_m0, double h0rc, double *beta, double *alpha,
                          double *s)
{
    if (!(a > 0.0 && a <= 1.0) || !(omega_m0 > 0.0 && omega_m0 <= 1.0) || !(h0rc > 0.0))
        return MG5_E_ARG;
    const double H0 = 100.0 / 299792.458;  // h/Mpc, c = 1
    const double a3 = a * a * a;
    const double E2 = omega_m0 / a3 + 1.0 - omega_m0;  // (H/H0)^2 of the LCDM-matched background
    const double E = std::sqrt(E2);
    const double hdot_h2 = -1.5 * (omega_m0 / a3) / E2;  // Hdot/H^2 = (1/2) dlnH^2/dlna
    const double b = 1.0 + 2.0 * (E * h0rc) * (1.0 + hdot_h2 / 3.0);
    const double rc = h0rc / H0;
    if (beta)
        *beta = b;
    if (alpha)
        *alpha = rc * rc / (3.0 * b * a * a);
    if (s)
        *s = omega_m0 * H0 * H0 / (b * a);
    return MG5_OK;
}

int mg5_workspace_bytes(int N, int precision, size_t *bytes)
{
    if (!bytes || check_size(N) != MG5_OK)
        return MG5_E_ARG;
    if (precision == MG5_FP64)
        *bytes = fp64_bytes(N);
    else if (precision == MG5_MIXED)
        *bytes = mixed_bytes(N);
    else
        return MG5_E_ARG;
    return MG5_OK;
}

int mg5_create(mg5_ctx **out, int device, size_t budget)
{
    if (!out)
        return MG5_E_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return MG5_E_CUDA;
    }
    if (device < 0 || device >= ndev)
        return MG5_E_ARG;
    mg5_ctx *ctx = new (std::nothrow) mg5_ctx();
    if (!ctx)
        return MG5_E_OOM;
    ctx->device = device;
    ctx->budget = budget;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess)
        e = alloc_partials(&ctx->partials);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&ctx->ls, sizeof(LevelScal) * kScalSlots);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&ctx->cnt, sizeof(SolveCounters));
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&ctx->h_rel, 64 * sizeof(double));
    if (e == cudaSuccess)
        e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&ctx->ev1);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&ctx->evb, cudaEventBlockingSync | cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = prepare_fused_kernels();
    if (e != cudaSuccess) {
        cudaGetLastError();
        mg5_destroy(ctx);
        return MG5_E_CUDA;
    }
    *out = ctx;
    return MG5_OK;
}

int mg5_release(mg5_ctx *ctx)
{
    if (!ctx)
        return MG5_E_ARG;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (Hier *h : ctx->hiers)
        free_hier(ctx, h);
    ctx->hiers.clear();
    for (MixedHier *m : ctx->mixed)
        free_mixed(m, &ctx->held);
    ctx->mixed.clear();
    for (PatchHier *ph : ctx->patches)
        free_patch(ctx, ph);
    ctx->patches.clear();
    free_batch(ctx);
    for (GraphEntry *g : ctx->graphs) {
        ctx->held -= g->bytes;
        graph_free(g);
    }
    ctx->graphs.clear();
    ctx_free(ctx, ctx->stage, ctx->stage_bytes);
    ctx->stage = nullptr;
    ctx->stage_bytes = 0;
    ctx_free(ctx, ctx->patch, ctx->patch_bytes);
    ctx->patch = nullptr;
    ctx->patch_bytes = 0;
    return MG5_OK;
}

int mg5_destroy(mg5_ctx *ctx)
{
    if (!ctx)
        return MG5_E_ARG;
    mg5_release(ctx);
    if (ctx->partials)
        cudaFree(ctx->partials);
    if (ctx->ls)
        cudaFree(ctx->ls);
    if (ctx->cnt)
        cudaFree(ctx->cnt);
    if (ctx->h_rel)
        cudaFreeHost(ctx->h_rel);
    if (ctx->ev0)
        cudaEventDestroy(ctx->ev0);
    if (ctx->ev1)
        cudaEventDestroy(ctx->ev1);
    if (ctx->evb)
        cudaEventDestroy(ctx->evb);
    ctx->prof.destroy();
    delete ctx;
    return MG5_OK;
}

const char *mg5_last_error(mg5_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t mg5_bytes_held(mg5_ctx *ctx) { return ctx ? ctx->held : 0; }

int mg5_set_autotune(mg5_ctx *ctx, int on)
{
    if (!ctx)
        return MG5_E_ARG;
    ctx->autotune = on != 0;
    return MG5_OK;
}

int mg5_autotune(mg5_ctx *ctx, int N, int precision, void *stream)
{
    if (!ctx || (precision != MG5_FP64 && precision != MG5_MIXED))
        return MG5_E_ARG;
    RET(check_size(N));
    CK(cudaSetDevice(ctx->device));
    return ctx_autotune(ctx, N, precision, (cudaStream_t)stream);
}

int mg5_set_blocking_wait(mg5_ctx *ctx, int on)
{
    if (!ctx)
        return MG5_E_ARG;
    ctx->blocking = on != 0;
    return MG5_OK;
}

int mg5_cached_bytes(mg5_ctx *ctx, int N, int precision, size_t *extra)
{
    if (!ctx || !extra)
        return MG5_E_ARG;
    RET(mg5_workspace_bytes(N, precision, extra));
    if (precision == MG5_FP64) {
        for (Hier *h : ctx->hiers)
            if (h->N == N)
                *extra = 0;
    } else {
        for (MixedHier *m : ctx->mixed)
            if (m->N == N)
                *extra = 0;
    }
    return MG5_OK;
}

int mg5_graph_workspace_bytes(int N, int with_grad, size_t *bytes)
{
    if (!bytes)
        return MG5_E_ARG;
    RET(check_size(N));
    *bytes = graph_entry_bytes(N, with_grad != 0);
    return MG5_OK;
}

int mg5_graph_cached_bytes(mg5_ctx *ctx, int N, const mg5_params *p, int with_grad, size_t *extra)
{
    if (!ctx || !p || !extra)
        return MG5_E_ARG;
    RET(check_size(N));
    *extra = p->precision == MG5_FP64 ? graph_entry_bytes64(N, with_grad != 0)
                                       : graph_entry_bytes(N, with_grad != 0);
    for (GraphEntry *g : ctx->graphs)
        if (!g->busy && g->N == N && g->grad == (with_grad != 0) && same_params(g->prm, *p) &&
            g->current())
            *extra = 0;
    return MG5_OK;
}

static const char *kProfNames[PK_COUNT] = {
    "sweep64", "resid_restrict64", "coarse_rhs64", "prolong64", "coarsest64",
    "sweep32", "resid_restrict32", "coarse_rhs32", "prolong32", "coarsest32",
    "resid64_mixed", "update_mixed", "patch_sweep64", "patch_resid64", "force64",
    "refine64", "reduce", "sweep64_coarse", "sweep32_coarse", "patch_sweep64_coarse"};

int mg5_profile_enable(mg5_ctx *ctx, int on)
{
    if (!ctx)
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    ctx->prof.resolve();
    ctx->prof.reset();
    ctx->prof.on = on != 0;
    return MG5_OK;
}

int mg5_profile_units(mg5_ctx *ctx, double *units, int n)
{
    if (!ctx || n < 0)
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    ctx->prof.resolve();
    for (int k = 0; k < n && k < PK_COUNT; ++k)
        units[k] = ctx->prof.units[k];
    return PK_COUNT;
}

int mg5_profile_read(mg5_ctx *ctx, double *ms, long long *calls, int n)
{
    if (!ctx || n < 0)
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaDeviceSynchronize());
    ctx->prof.resolve();
    for (int k = 0; k < n && k < PK_COUNT; ++k) {
        if (ms)
            ms[k] = ctx->prof.ms[k];
        if (calls)
            calls[k] = ctx->prof.calls[k];
    }
    return PK_COUNT;
}

const char *mg5_profile_name(int k) { return (k >= 0 && k < PK_COUNT) ? kProfNames[k] : ""; }

int mg5_solve_fifth_force(mg5_ctx *ctx, const double *delta, int N, const mg5_params *p,
                          unsigned flags, double *phi, double *grad, mg5_info *info, void *stream)
{
    if (!ctx || !delta || !phi)
        return MG5_E_ARG;
    RET(check_size(N));
    RET(check_params(p));
    if (flags & ~(MG5_WARM | MG5_HOST_IO | MG5_FMG | MG5_GRAPH))
        return MG5_E_ARG;
    if ((flags & MG5_GRAPH) && (flags & MG5_WARM))
        return MG5_E_ARG;
    if ((flags & MG5_GRAPH) && p->precision == MG5_FP64) {
        int sz[kMaxLevels];
        if (num_levels(N, sz) < 2 || (p->nu1 + p->nu2) % 2) {
            ctx->err = "MG5_GRAPH with MG5_FP64 needs two grids or more and nu1 + nu2 even";
            return MG5_E_ARG;
        }
    }
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (info)
        std::memset(info, 0, sizeof(*info));
    const long long n3 = (long long)N * N * N;
    const size_t fb = (size_t)n3 * sizeof(double);
    const double *d_delta = delta;
    double *d_phi = phi, *d_grad = grad;
    if (ctx->autotune)
        RET(ctx_autotune(ctx, N, p->precision, st));
    CK(cudaEventRecord(ctx->ev0, st));
    if (flags & MG5_HOST_IO) {
        RET(ensure_buffer(ctx, &ctx->stage, &ctx->stage_bytes, fb * (grad ? 5 : 2)));
        d_phi = ctx->stage;
        double *dd = ctx->stage + n3;
        d_grad = grad ? ctx->stage + 2 * n3 : nullptr;
        CK(cudaMemcpyAsync(dd, delta, fb, cudaMemcpyHostToDevice, st));
        d_delta = dd;
        if (flags & MG5_WARM)
            CK(cudaMemcpyAsync(d_phi, phi, fb, cudaMemcpyHostToDevice, st));
    }
    if (!(flags & MG5_WARM))
        CK(cudaMemsetAsync(d_phi, 0, fb, st));
    int status;
    if (flags & MG5_GRAPH) {
        status = solve_graph(ctx, d_delta, N, p, d_phi, d_grad, (flags & MG5_FMG) != 0, info, st);
        if (status == MG5_E_CUDA || status == MG5_E_ARG || status == MG5_E_OOM)
            return status;
        if (flags & MG5_HOST_IO) {
            CK(cudaMemcpyAsync(phi, d_phi, fb, cudaMemcpyDeviceToHost, st));
            if (grad)
                CK(cudaMemcpyAsync(grad, d_grad, 3 * fb, cudaMemcpyDeviceToHost, st));
        }
        CK(cudaEventRecord(ctx->ev1, st));
        CK(ctx_wait(ctx, st));
        if (info) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
            info->ms_total = ms;
            info->status = status;
        }
        return status;
    }
    if (p->precision == MG5_FP64) {
        status = solve64(ctx, d_delta, N, p, d_phi, (flags & MG5_WARM) != 0, (flags & MG5_FMG) != 0,
                         info, st);
    } else {
        MixedHier *mh = nullptr;
        for (MixedHier *m : ctx->mixed)
            if (m->N == N)
                mh = m;
        if (!mh) {
            int rc = alloc_mixed(N, ctx->budget, &ctx->held, &mh, &ctx->err);
            if (rc != MG5_OK)
                return rc;
            ctx->mixed.push_back(mh);
        }
        MixedShared sh{ctx->partials, ctx->ls, ctx->cnt, ctx->h_rel, &ctx->prof,
                       ctx->blocking ? ctx->evb : nullptr};
        status = solve_mixed(mh, sh, d_delta, p, d_phi, info, st, &ctx->err, !(flags & MG5_WARM));
    }
    if (status == MG5_E_CUDA || status == MG5_E_ARG || status == MG5_E_OOM)
        return status;
    if (d_grad) {
        ProfScope ps(&ctx->prof, PK_FORCE, st, (double)n3);
        CK(launch_force(d_phi, N, N, N, 0, p->h, 1, d_grad, st));
    }
    if (flags & MG5_HOST_IO) {
        CK(cudaMemcpyAsync(phi, d_phi, fb, cudaMemcpyDeviceToHost, st));
        if (grad)
            CK(cudaMemcpyAsync(grad, d_grad, 3 * fb, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaEventRecord(ctx->ev1, st));
    SolveCounters cnt;
    CK(cudaMemcpyAsync(&cnt, ctx->cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    double tail[2];
    CK(cudaMemcpyAsync(tail, &ctx->ls[0].c, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(tail + 1, &ctx->ls[0].mean, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(ctx_wait(ctx, st));
    ctx->prof.resolve();
    if (status == MG5_OK && cnt.clamped > 0)
        status = MG5_W_DISC_CLAMP;
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        info->ms_total = ms;
        info->status = status;
        info->disc_clamped = (long long)cnt.clamped;
        info->compat_c = tail[0];
        info->phi_mean_removed = tail[1];
        const long long nc = info->coarsest_n;
        info->cell_updates += (long long)cnt.coarse_sweeps * nc * nc * nc;
        info->coarse_sweeps = cnt.coarse_sweeps;
    }
    return status;
}

int mg5_force(mg5_ctx *ctx, const double *phi, const int dims[3], int ghost, double h, int periodic,
              double *grad, void *stream)
{
    if (!ctx || !phi || !dims || !grad || !(h > 0.0) || ghost < 0)
        return MG5_E_ARG;
    for (int a = 0; a < 3; ++a)
        if (dims[a] - 2 * ghost < 1)
            return MG5_E_ARG;
    if (periodic && ghost != 0)
        return MG5_E_ARG;
    if (!periodic && ghost < 1)
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    ProfScope ps(&ctx->prof, PK_FORCE, (cudaStream_t)stream,
                 (double)(dims[0] - 2 * ghost) * (dims[1] - 2 * ghost) * (dims[2] - 2 * ghost));
    CK(launch_force(phi, dims[0], dims[1], dims[2], ghost, h, periodic ? 1 : 0, grad,
                    (cudaStream_t)stream));
    return MG5_OK;
}

int mg5_refine_interpolate(mg5_ctx *ctx, const double *phic, int Nc, const int o[3], const int pn[3],
                           int ghost, double *fine, void *stream)
{
    if (!ctx || !phic || !o || !pn || !fine || Nc < 1 || ghost < 0 || ghost > 4)
        return MG5_E_ARG;
    for (int a = 0; a < 3; ++a)
        if (o[a] < 0 || o[a] >= Nc || pn[a] < 1 || pn[a] > Nc)
            return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    ProfScope ps(&ctx->prof, PK_REFINE, (cudaStream_t)stream,
                 (double)(2 * pn[0] + 2 * ghost) * (2 * pn[1] + 2 * ghost) * (2 * pn[2] + 2 * ghost));
    CK(launch_refine(phic, Nc, o, pn, ghost, fine, (cudaStream_t)stream));
    return MG5_OK;
}

int mg5_refine_interpolate_cubic(mg5_ctx *ctx, const double *phic, int Nc, const int o[3],
                                 const int pn[3], int ghost, double *fine, void *stream)
{
    if (!ctx || !phic || !o || !pn || !fine || Nc < 4 || ghost < 0 || ghost > 4)
        return MG5_E_ARG;
    for (int a = 0; a < 3; ++a)
        if (o[a] < 0 || o[a] >= Nc || pn[a] < 1 || pn[a] > Nc)
            return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    ProfScope ps(&ctx->prof, PK_REFINE, (cudaStream_t)stream,
                 (double)(2 * pn[0] + 2 * ghost) * (2 * pn[1] + 2 * ghost) * (2 * pn[2] + 2 * ghost));
    CK(launch_refine_cubic(phic, Nc, o, pn, ghost, fine, (cudaStream_t)stream));
    return MG5_OK;
}

static int floor_div4(int x) { return x >= 0 ? x / 4 : -((-x + 3) / 4); }



int mg5_refine_interpolate_box(mg5_ctx *ctx, const double *box, const int bd[3], int pg,
                               const int o[3], const int pn[3], int ghost, double *fine,
                               void *stream)
{
    if (!ctx || !box || !bd || !o || !pn || !fine || pg < 0 || ghost < 0 || ghost > 4)
        return MG5_E_ARG;
    for (int a = 0; a < 3; ++a) {
        const int D = bd[a] - 2 * pg;
        if (D < 1 || o[a] < 0 || pn[a] < 1 || o[a] + pn[a] > D)
            return MG5_E_ARG;
        // every coarse centre the trilinear stencil touches must lie in the box
        const int lo = floor_div4(4 * o[a] - 2 * ghost - 1);
        const int hi = floor_div4(4 * o[a] + 2 * (2 * pn[a] + ghost - 1) - 1) + 1;
        if (lo + pg < 0 || hi + pg > bd[a] - 1) {
            ctx->err = "refine_interpolate_box: the window and its fine ghosts reach outside the box";
            return MG5_E_ARG;
        }
    }
    CK(cudaSetDevice(ctx->device));
    ProfScope ps(&ctx->prof, PK_REFINE, (cudaStream_t)stream,
                 (double)(2 * pn[0] + 2 * ghost) * (2 * pn[1] + 2 * ghost) * (2 * pn[2] + 2 * ghost));
    CK(launch_refine_box(box, bd, pg, o, pn, ghost, fine, (cudaStream_t)stream));
    return MG5_OK;
}

namespace {

// FAS V-cycles on the Dirichlet patch hierarchy (ghost shells fixed).
struct RunPatch {
    mg5_ctx *ctx;
    PatchHier *h;
    const mg5_params *p;
    cudaStream_t st;
    double hl[kMaxLevels];
    long long cu = 0;
    // device scratch: the context's (its patch slot), or a captured graph's own
    LevelScal *lsp = nullptr;
    SolveCounters *cntb = nullptr;
    double2 *partb = nullptr;
    // masked relaxation (Sec. 3.3): the caller's mask on grid 0, its restrictions below
    const unsigned char *mk[kMaxLevels] = {};

    void bind_ctx_scratch()
    {
        lsp = ctx->ls + kPatchSlot;
        cntb = ctx->cnt;
        partb = ctx->partials;
    }
    bool bound() const { return lsp && cntb && partb; }

    // extrapolation weight of the coarse ghosts on grid l >= 1 (see k_patch.cu)
    static double ghost_w(int l)
    {
        const double a = (double)(1 << (l - 1));
        return -(a - 0.5) / (a + 0.5);
    }

    int sweep(int l)
    {
        mg5_ctx *ctx = this->ctx;
        const double cells = (double)int_cells(h->q[l]);
        {
            ProfScope ps(&ctx->prof, l == 0 ? PK_PATCH_SWEEP : PK_PATCH_SWEEPC, st, cells);
            CK(launch_patch_sweep(h->v[l], h->tmp[l], h->f[l], 0.0, h->q[l],
                                  make_coef<double>(hl[l], p->alpha, omega_of(p)), &cntb->clamped, st,
                                  l > 0 ? h->v0[l] : nullptr, l > 0 ? ghost_w(l) : 0.0, mk[l]));
        }
        std::swap(h->v[l], h->tmp[l]);
        cu += (long long)cells;
        return MG5_OK;
    }

    int coarsest(int l)
    {
        mg5_ctx *ctx = this->ctx;
        ProfScope ps(&ctx->prof, PK_COARSEST64, st);
        CK(launch_pbox_coarsest(h->v[l], h->tmp[l], h->f[l], h->q[l],
                                make_coef<double>(hl[l], p->alpha, omega_of(p)), p->nu_coarse, kCoarseRtol,
                                &cntb->clamped, &cntb->coarse_sweeps, st,
                                l > 0 ? h->v0[l] : nullptr, l > 0 ? ghost_w(l) : 0.0, mk[l]));
        return MG5_OK;
    }

    int resid_restrict(int l, bool finalize)
    {
        mg5_ctx *ctx = this->ctx;
        int nb = 0;
        {
            ProfScope ps(&ctx->prof, PK_PATCH_RESID, st, (double)int_cells(h->q[l]));
            CK(launch_pbox_resid_restrict(h->v[l], h->f[l], h->q[l],
                                          make_coef<double>(hl[l], p->alpha), h->v[l + 1],
                                          h->v0[l + 1], h->f[l + 1], partb, &nb, st, mk[l],
                                          Fin{finalize ? lsp : nullptr, FIN_NORM,
                                              (double)int_cells(h->q[l])}));
        }
        return MG5_OK;
    }

    int coarse_visit(int l)
    {
        mg5_ctx *ctx = this->ctx;
        // v = v0 on entry, its ghosts reset to the fixed coarse values by the restriction
        CK(launch_pbox_coarse_rhs(h->v[l], h->f[l], h->q[l], make_coef<double>(hl[l], p->alpha), st));
        if (l == h->nlev - 1)
            return coarsest(l);
        for (int s = 0; s < p->nu1; ++s)
            RET(sweep(l));
        RET(resid_restrict(l, false));
        RET(coarse_visit(l + 1));
        CK(launch_pbox_prolong(h->v[l + 1], h->v0[l + 1], h->q[l + 1], h->v[l], st, mk[l]));
        for (int s = 0; s < p->nu2; ++s)
            RET(sweep(l));
        return MG5_OK;
    }
};

}  // namespace

constexpr double kMaskGsFraction = 0.1;   // masked fraction below which sweeps go first
constexpr int kMaskGsCheck = 4;            // sweeps between residual checks
constexpr int kMaskGsMax = 64;             // sweeps before V-cycles take over

// The host-driven patch relaxation; mask (device, interior-indexed) or nullptr for every cell.
static int relax_patch_impl(mg5_ctx *ctx, const double *delta_f, const int pf[3],
                            const unsigned char *mask, const mg5_params *p, double compat_c,
                            double *phi, mg5_info *info, void *stream)
{
    if (!ctx || !delta_f || !pf || !phi)
        return MG5_E_ARG;
    RET(check_params(p));
    for (int a = 0; a < 3; ++a)
        if (pf[a] < 2 || (pf[a] & 1))
            return MG5_E_ARG;
    if (!std::isfinite(compat_c))
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (info)
        std::memset(info, 0, sizeof(*info));
    PatchHier *h = nullptr;
    RET(get_patch(ctx, pf, &h));
    if (mask)
        RET(get_patch_masks(ctx, h));
    const long long ni = (long long)int_cells(pf);
    const long long nbox = (long long)box_cells(pf);
    CK(cudaEventRecord(ctx->ev0, st));
    LevelScal *ls = ctx->ls + kPatchSlot;
    CK(cudaMemsetAsync(ls, 0, sizeof(LevelScal), st));
    CK(cudaMemsetAsync(ctx->cnt, 0, sizeof(SolveCounters), st));
    int nb = 0;
    // f0 = s delta + c; the tolerance is relative to ||s delta|| (over the masked cells)
    if (mask) {
        CK(launch_scale_masked(delta_f, p->s, h->f[0], ni, mask, ctx->partials, &nb, st, compat_c));
        for (int l = 1; l < h->nlev; ++l)
            CK(launch_mask_restrict(l == 1 ? mask : h->mk[l - 1], h->q[l - 1], h->mk[l], st));
        CK(launch_finalize(ctx->partials, nb, (double)ni, ls, FIN_FNORM, st));
    } else {
        CK(launch_scale(delta_f, p->s, h->f[0], ni, ctx->partials, &nb, st, compat_c, nullptr,
                        Fin{ls, FIN_FNORM, (double)ni}));
    }
    double masked_fraction = 1.0;
    if (mask) {
        CK(launch_finalize(ctx->partials, nb, (double)ni, ls, FIN_MEAN, st));   // mean = fraction
        CK(cudaMemcpyAsync(ctx->h_rel, &ls->mean, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(ctx_wait(ctx, st));
        masked_fraction = *ctx->h_rel;
    }
    // the ping-pong partner of the caller's box carries the same ghost shell
    CK(cudaMemcpyAsync(h->tmp[0], phi, nbox * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int l = 1; l < h->nlev; ++l)
        CK(launch_pbox_ghosts(l == 1 ? phi : h->v[l - 1], h->q[l - 1], h->v[l], h->tmp[l], h->v0[l],
                              st));
    struct Restore {
        PatchHier *h;
        double *own;
        ~Restore()
        {
            h->v[0] = nullptr;
            h->tmp[0] = own;
        }
    } restore{h, h->tmp[0]};
    h->v[0] = phi;
    RunPatch R{ctx, h, p, st, {}, 0};
    R.bind_ctx_scratch();
    if (!R.bound()) {
        ctx->err = "relax_patch: context scratch not allocated";
        return MG5_E_ARG;
    }
    if (mask) {
        R.mk[0] = mask;
        for (int l = 1; l < h->nlev; ++l)
            R.mk[l] = h->mk[l];
    }
    for (int l = 0; l < h->nlev; ++l)
        R.hl[l] = p->h * (double)(1 << l);
    int status = MG5_E_NOT_CONVERGED;
    double best = INFINITY;
    int cyc = 0, nh = 0;
    auto record = [&](double rel) {
        if (info) {
            info->rel_residual = rel;
            if (nh < 64) {
                info->history[nh] = rel;
                info->n_history = nh + 1;
            }
        }
        ++nh;
    };
    // A sparse mask (Sec. 3.3's criterion deep in a hierarchy) leaves small clusters of cells
    // between fixed values, where masked sweeps alone converge in tens of sweeps: try those
    // first (checked every kMaskGsCheck sweeps, at most kMaskGsMax), then V-cycles from there.
    bool done = false;
    if (mask && masked_fraction < kMaskGsFraction) {
        const CoefT<double> cf0 = make_coef<double>(p->h, p->alpha);
        for (int gs = 0;;) {
            CK(launch_patch_residual(h->v[0], h->f[0], 0.0, pf, cf0, ctx->partials, &nb, st, mask,
                                     Fin{ls, FIN_NORM, (double)ni}));
            CK(cudaMemcpyAsync(ctx->h_rel, &ls->rel, sizeof(double), cudaMemcpyDeviceToHost, st));
            CK(ctx_wait(ctx, st));
            const double rel = *ctx->h_rel;
            record(rel);
            if (!std::isfinite(rel) || rel <= p->tol) {
                status = std::isfinite(rel) ? MG5_OK : MG5_E_NONFINITE;
                done = true;
                break;
            }
            if (gs >= kMaskGsMax)
                break;
            for (int k = 0; k < kMaskGsCheck; ++k, ++gs)
                RET(R.sweep(0));
        }
    }
    for (; !done; ++cyc) {
        if (h->nlev == 1) {
            RET(R.coarsest(0));
            CK(launch_patch_residual(h->v[0], h->f[0], 0.0, pf, make_coef<double>(p->h, p->alpha),
                                     ctx->partials, &nb, st, mask, Fin{ls, FIN_NORM, (double)ni}));
        } else {
            for (int s = 0; s < p->nu1; ++s)
                RET(R.sweep(0));
            RET(R.resid_restrict(0, true));
        }
        CK(cudaMemcpyAsync(ctx->h_rel, &ls->rel, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(ctx_wait(ctx, st));
        const double rel = *ctx->h_rel;
        record(rel);
        if (!std::isfinite(rel)) {
            status = MG5_E_NONFINITE;
            break;
        }
        if (rel <= p->tol) {
            status = MG5_OK;
            break;
        }
        best = std::min(best, rel);
        if (cyc >= 3 && rel > 10.0 * best) {
            status = MG5_E_DIVERGED;
            break;
        }
        if (cyc >= p->max_cycles)
            break;
        if (h->nlev == 1)
            continue;
        RET(R.coarse_visit(1));
        CK(launch_pbox_prolong(h->v[1], h->v0[1], h->q[1], h->v[0], st, mask));
        for (int s = 0; s < p->nu2; ++s)
            RET(R.sweep(0));
    }
    if (h->v[0] != phi)
        CK(cudaMemcpyAsync(phi, h->v[0], nbox * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaEventRecord(ctx->ev1, st));
    SolveCounters cnt;
    CK(cudaMemcpyAsync(&cnt, ctx->cnt, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    CK(ctx_wait(ctx, st));
    ctx->prof.resolve();
    if (status == MG5_OK && cnt.clamped > 0)
        status = MG5_W_DISC_CLAMP;
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        info->ms_total = ms;
        info->status = status;
        info->cycles = cyc;
        info->levels = h->nlev;
        info->coarsest_n = h->q[h->nlev - 1][0];
        info->cell_updates = R.cu + (long long)cnt.coarse_sweeps * (long long)int_cells(h->q[h->nlev - 1]);
        info->coarse_sweeps = cnt.coarse_sweeps;
        info->disc_clamped = (long long)cnt.clamped;
        info->compat_c = compat_c;
    }
    return status;
}

int mg5_relax_patch(mg5_ctx *ctx, const double *delta_f, const int pf[3], const mg5_params *p,
                    double compat_c, double *phi, mg5_info *info, void *stream)
{
    return relax_patch_impl(ctx, delta_f, pf, nullptr, p, compat_c, phi, info, stream);
}

int mg5_relax_patch_masked(mg5_ctx *ctx, const double *delta_f, const int pf[3],
                           const unsigned char *mask, const mg5_params *p, double compat_c,
                           double *phi, mg5_info *info, void *stream)
{
    if (!mask)
        return MG5_E_ARG;
    return relax_patch_impl(ctx, delta_f, pf, mask, p, compat_c, phi, info, stream);
}

int mg5_parent_force_mask(mg5_ctx *ctx, const double *grad_phi, const double *grad_gr,
                          const int pd[3], int periodic, const int o[3], const int pn[3],
                          double theta, unsigned char *mask, long long *count, void *stream)
{
    if (!ctx || !grad_phi || !grad_gr || !pd || !o || !pn || !mask || !(theta >= 0.0) ||
        !std::isfinite(theta))
        return MG5_E_ARG;
    for (int a = 0; a < 3; ++a) {
        if (pd[a] < 1 || pn[a] < 1 || o[a] < 0)
            return MG5_E_ARG;
        if (periodic ? (o[a] >= pd[a] || pn[a] > pd[a]) : ((long long)o[a] + pn[a] > pd[a]))
            return MG5_E_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *dcount = nullptr;
    if (count) {
        // every solve of this context synchronises before it returns, and a context serves one
        // host thread at a time: between calls its counters and pinned scalars are free
        dcount = &ctx->cnt->clamped;
        CK(cudaMemsetAsync(dcount, 0, sizeof(*dcount), st));
    }
    CK(launch_parent_force_mask(grad_phi, grad_gr, pd, periodic, o, pn, theta, mask, dcount, st));
    if (count) {
        CK(cudaMemcpyAsync(ctx->h_rel, dcount, sizeof(*dcount), cudaMemcpyDeviceToHost, st));
        CK(ctx_wait(ctx, st));
        unsigned long long c = 0;
        std::memcpy(&c, ctx->h_rel, sizeof(c));
        *count = (long long)c;
    }
    return MG5_OK;
}

static size_t patch_entry_bytes(const int pf[3], size_t hier_bytes)
{
    return hier_bytes + (box_cells(pf) + int_cells(pf)) * sizeof(double) +
           sizeof(double2) * kMaxPartials + sizeof(LevelScal) * kScalSlots + sizeof(SolveCounters) +
           sizeof(BoxCtl) + sizeof(double);
}

// The patch relaxation as one graph: f = s delta + c (c read on the device), the coarse ghost
// shells from the entry's box, the first smoothing and check, then the V-cycle as a WHILE node
// (body: coarse-grid correction, post- and next pre-smoothing, check).  As for the periodic FP64
// graph the body swaps each grid's buffers nu1 + nu2 times (even).
static int capture_patch(mg5_ctx *ctx, GraphEntry *g, const mg5_params *p, cudaStream_t st,
                         cudaStream_t body_st);

}  // extern "C"

namespace {

int capture_patch_impl(mg5_ctx *ctx, GraphEntry *g, const mg5_params *p, cudaStream_t st,
                       cudaStream_t body_st)
{
    PatchHier *h = g->hierp;
    const int *pf = g->pdims;
    const long long ni = (long long)int_cells(pf), nbox = (long long)box_cells(pf);
    RunPatch R{ctx, h, p, st, {}, 0};
    R.lsp = g->ls;
    R.cntb = g->cnt;
    R.partb = g->partials;
    if (!R.bound() || !g->ctl || !g->phi || !g->delta || !g->cdev) {
        ctx->err = "capture_patch: entry scratch not allocated";
        return MG5_E_ARG;
    }
    for (int l = 0; l < h->nlev; ++l)
        R.hl[l] = p->h * (double)(1 << l);
    const long long L0 = launches_total();
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) {
        ctx->err = "capture_patch: stream is not capturing";
        return MG5_E_ARG;
    }
    cudaGraphConditionalHandle hnd;
    CK(cudaGraphConditionalHandleCreate(&hnd, graph, 0, cudaGraphCondAssignDefault));
    CK(launch_ctl_init(g->ctl, p->tol, p->max_cycles, st));
    CK(cudaMemsetAsync(g->ls, 0, sizeof(LevelScal) * kScalSlots, st));
    CK(cudaMemsetAsync(g->cnt, 0, sizeof(SolveCounters), st));
    int nb = 0;
    CK(launch_scale(g->delta, p->s, h->f[0], ni, g->partials, &nb, st, 0.0, g->cdev,
                    Fin{g->ls, FIN_FNORM, (double)ni}));
    CK(cudaMemcpyAsync(h->tmp[0], g->phi, nbox * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int l = 1; l < h->nlev; ++l)
        CK(launch_pbox_ghosts(l == 1 ? g->phi : h->v[l - 1], h->q[l - 1], h->v[l], h->tmp[l],
                              h->v0[l], st));
    h->v[0] = g->phi;
    for (int k = 0; k < p->nu1; ++k)
        RET(R.sweep(0));
    RET(R.resid_restrict(0, true));
    CK(launch_loop_check(g->ls, g->ctl, hnd, st));
    const long long cells_fixed = R.cu;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    const long long L1 = launches_total();
    CK(cudaStreamBeginCaptureToGraph(body_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    double *const v0_start = h->v[0];
    RunPatch B = R;
    B.st = body_st;
    B.cu = 0;
    int rc = B.coarse_visit(1);
    if (rc == MG5_OK && launch_pbox_prolong(h->v[1], h->v0[1], h->q[1], h->v[0], body_st) != cudaSuccess)
        rc = MG5_E_CUDA;
    for (int k = 0; k < p->nu2 && rc == MG5_OK; ++k)
        rc = B.sweep(0);
    for (int k = 0; k < p->nu1 && rc == MG5_OK; ++k)
        rc = B.sweep(0);
    if (rc == MG5_OK)
        rc = B.resid_restrict(0, true);
    if (rc == MG5_OK && launch_loop_check(g->ls, g->ctl, hnd, body_st) != cudaSuccess)
        rc = MG5_E_CUDA;
    cudaGraph_t g_out = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(body_st, &g_out);
    RET(rc);
    CK(e_end);
    if (h->v[0] != v0_start) {
        ctx->err = "capture_patch: the loop body does not return the grids to their buffers";
        return MG5_E_ARG;
    }
    const long long L2 = launches_total();
    if (h->v[0] != g->phi)
        CK(cudaMemcpyAsync(g->phi, h->v[0], nbox * sizeof(double), cudaMemcpyDeviceToDevice, st));
    g->stats.launches_fixed = (L1 - L0) + (launches_total() - L2);
    g->stats.launches_per_iter = L2 - L1;
    g->stats.cells_per_iter = B.cu;
    g->stats.cells_fixed = cells_fixed;
    g->stats.inner = 1;
    return MG5_OK;
}

}  // namespace

extern "C" {

static int capture_patch(mg5_ctx *ctx, GraphEntry *g, const mg5_params *p, cudaStream_t st,
                         cudaStream_t body_st)
{
    return capture_patch_impl(ctx, g, p, st, body_st);
}

int mg5_relax_patch_graph(mg5_ctx *ctx, const double *delta_f, const int pf[3], const mg5_params *p,
                          double compat_c, double *phi, mg5_info *info, void *stream)
{
    if (!ctx || !delta_f || !pf || !phi)
        return MG5_E_ARG;
    RET(check_params(p));
    for (int a = 0; a < 3; ++a)
        if (pf[a] < 2 || (pf[a] & 1))
            return MG5_E_ARG;
    if (!std::isfinite(compat_c))
        return MG5_E_ARG;
    int q[kMaxLevels][3];
    if (patch_levels(pf, q) < 2 || (p->nu1 + p->nu2) % 2) {
        ctx->err = "relax_patch_graph needs two grids or more and nu1 + nu2 even";
        return MG5_E_ARG;
    }
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (info)
        std::memset(info, 0, sizeof(*info));
    const long long ni = (long long)int_cells(pf), nbox = (long long)box_cells(pf);
    // the cached entry for (pf, params), or a new capture
    GraphEntry *g = nullptr;
    for (GraphEntry *x : ctx->graphs)
        if (!x->busy && x->hierp && x->pdims[0] == pf[0] && x->pdims[1] == pf[1] &&
            x->pdims[2] == pf[2] && same_params(x->prm, *p)) {
            g = x;
            break;
        }
    if (!g) {
        while (ctx->graphs.size() >= kGraphCacheMax) {
            GraphEntry *v = graph_take_idle(ctx);
            if (!v)
                break;
            graph_free(v);
        }
        g = new GraphEntry();
        g->prm = *p;
        for (int a = 0; a < 3; ++a)
            g->pdims[a] = pf[a];
        cudaError_t e = alloc_patch_raw(pf, &g->hierp);
        const size_t need = patch_entry_bytes(pf, g->hierp ? g->hierp->bytes : 0);
        if (e == cudaSuccess && ctx->budget && ctx->held + need > ctx->budget)
            e = cudaErrorMemoryAllocation;
        for (void **q2 : {(void **)&g->partials, (void **)&g->ls, (void **)&g->cnt, (void **)&g->ctl,
                          (void **)&g->delta, (void **)&g->phi, (void **)&g->cdev}) {
            if (e != cudaSuccess)
                break;
            size_t b = q2 == (void **)&g->partials ? sizeof(double2) * kMaxPartials
                     : q2 == (void **)&g->ls       ? sizeof(LevelScal) * kScalSlots
                     : q2 == (void **)&g->cnt      ? sizeof(SolveCounters)
                     : q2 == (void **)&g->ctl      ? sizeof(BoxCtl)
                     : q2 == (void **)&g->delta    ? ni * sizeof(double)
                     : q2 == (void **)&g->phi      ? nbox * sizeof(double)
                                                   : sizeof(double);
            e = cudaMalloc(q2, b);
        }
        if (e == cudaSuccess)
            e = cudaMemset(g->partials, 0, sizeof(double2) * kMaxPartials);
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&g->rb, sizeof(GraphReadback));
        g->bytes = need;
        cudaStream_t origin = nullptr, body = nullptr;
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking);
        int rc = e == cudaSuccess ? MG5_OK : (e == cudaErrorMemoryAllocation ? MG5_E_OOM : MG5_E_CUDA);
        if (rc != MG5_OK)
            ctx->err = std::string("relax_patch_graph: ") + cudaGetErrorString(e);
        const long long l0 = launches_total();
        const bool prof_on = ctx->prof.on;
        if (rc == MG5_OK) {
            ctx->prof.on = false;
            e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                rc = capture_patch(ctx, g, p, origin, body);
                cudaGraph_t graph = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
                if (rc == MG5_OK && e2 == cudaSuccess) {
                    g->graph = graph;
                    e = cudaGraphInstantiate(&g->exec, graph, 0);
                } else {
                    if (graph)
                        cudaGraphDestroy(graph);
                    if (e2 != cudaSuccess)
                        e = e2;
                }
            }
            ctx->prof.on = prof_on;
            count_launch(l0 - launches_total());
            if (rc == MG5_OK && e != cudaSuccess) {
                ctx->err = std::string("relax_patch_graph: ") + cudaGetErrorString(e);
                rc = MG5_E_CUDA;
            }
        }
        if (origin)
            cudaStreamDestroy(origin);
        if (body)
            cudaStreamDestroy(body);
        cudaGetLastError();
        if (rc != MG5_OK) {
            graph_free(g);
            return rc;
        }
        graph_insert(ctx, g);
    } else {
        g->busy = true;
        g->last_use = ++ctx->graph_clock;
    }
    CK(cudaEventRecord(ctx->ev0, st));
    g->rb->c_in = compat_c;
    int rc = MG5_OK;
    cudaError_t e = cudaMemcpyAsync(g->cdev, &g->rb->c_in, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->delta, delta_f, ni * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->phi, phi, nbox * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaGraphLaunch(g->exec, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(phi, g->phi, nbox * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&g->rb->ctl, g->ctl, sizeof(BoxCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&g->rb->cnt, g->cnt, sizeof(SolveCounters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&g->rb->ls0, g->ls, sizeof(LevelScal), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaEventRecord(ctx->ev1, st);
    if (e == cudaSuccess)
        e = ctx_wait(ctx, st);
    if (e != cudaSuccess) {
        ctx->err = std::string("relax_patch_graph: ") + cudaGetErrorString(e);
        cudaGetLastError();
        graph_checkin(g);
        return MG5_E_CUDA;
    }
    rc = graph_finish(g, info);
    if (info) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        info->ms_total = ms;
        info->compat_c = compat_c;
    }
    return rc;
}

static bool same_params(const mg5_params &a, const mg5_params &b)
{
    return std::memcmp(&a, &b, sizeof(mg5_params)) == 0;
}

}  // extern "C"

namespace mg5 {

size_t graph_bytes(int N, int precision, bool grad)
{
    return precision == MG5_FP64 ? graph_entry_bytes64(N, grad) : graph_entry_bytes(N, grad);
}

size_t graph_held(mg5_ctx *ctx)
{
    size_t t = 0;
    for (GraphEntry *g : ctx->graphs)
        t += g->bytes;
    return t;
}

GraphEntry *graph_checkout(mg5_ctx *ctx, int N, const mg5_params *p, bool grad)
{
    for (GraphEntry *g : ctx->graphs)
        if (!g->busy && g->N == N && g->grad == grad && same_params(g->prm, *p) && g->current()) {
            g->busy = true;
            g->last_use = ++ctx->graph_clock;
            return g;
        }
    return nullptr;
}

int graph_count(mg5_ctx *ctx, int N, const mg5_params *p, bool grad)
{
    int c = 0;
    for (GraphEntry *g : ctx->graphs)
        c += g->N == N && g->grad == grad && same_params(g->prm, *p) && g->current();
    return c;
}

void graph_insert(mg5_ctx *ctx, GraphEntry *g)
{
    g->busy = true;
    g->last_use = ++ctx->graph_clock;
    ctx->graphs.push_back(g);
    ctx->held += g->bytes;
}

GraphEntry *graph_take_idle(mg5_ctx *ctx)
{
    auto best = ctx->graphs.end();
    for (auto it = ctx->graphs.begin(); it != ctx->graphs.end(); ++it)
        if (!(*it)->busy && (best == ctx->graphs.end() || (*it)->last_use < (*best)->last_use))
            best = it;
    if (best == ctx->graphs.end())
        return nullptr;
    GraphEntry *g = *best;
    ctx->graphs.erase(best);
    ctx->held -= g->bytes;
    return g;
}

void graph_free(GraphEntry *g)
{
    if (g->exec)
        cudaGraphExecDestroy(g->exec);
    if (g->graph)
        cudaGraphDestroy(g->graph);
    size_t hb = 0;
    if (g->hier)
        free_mixed(g->hier, &hb);
    free_hier_raw(g->hier64);
    free_patch_raw(g->hierp);
    if (g->cdev)
        cudaFree(g->cdev);
    for (void *p : {(void *)g->partials, (void *)g->ls, (void *)g->cnt, (void *)g->ctl,
                    (void *)g->delta, (void *)g->phi, (void *)g->gout})
        if (p)
            cudaFree(p);
    if (g->rb)
        cudaFreeHost(g->rb);
    delete g;
}

int graph_build(int device, int N, const mg5_params *p, bool grad, GraphEntry **out,
                std::string *err)
{
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        *err = "graph solve: cannot select the device";
        return MG5_E_CUDA;
    }
    GraphEntry *g = new GraphEntry();
    g->N = N;
    g->prm = *p;
    g->grad = grad;
    g->sched = schedule_version();   // read before the capture reads the schedules
    size_t hb = 0;
    int rc = alloc_mixed(N, 0, &hb, &g->hier, err);
    const size_t n3 = (size_t)N * N * N;
    cudaError_t e = rc == MG5_OK ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
        e = alloc_partials(&g->partials);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->ls, sizeof(LevelScal) * kScalSlots);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->cnt, sizeof(SolveCounters));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->ctl, sizeof(BoxCtl));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->delta, n3 * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->phi, n3 * sizeof(double));
    if (e == cudaSuccess && grad)
        e = cudaMalloc((void **)&g->gout, 3 * n3 * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&g->rb, sizeof(GraphReadback));
    g->bytes = graph_entry_bytes(N, grad);
    cudaStream_t origin = nullptr, body = nullptr;
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking);
    const long long l0 = launches_total();
    if (e == cudaSuccess) {
        e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            MixedShared sh{g->partials, g->ls, g->cnt, nullptr, nullptr};
            rc = capture_mixed(g->hier, sh, g->delta, p, g->phi, g->gout, g->ctl, origin, body,
                               &g->stats, err);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
            if (rc == MG5_OK && e2 == cudaSuccess) {
                g->graph = graph;
                e = cudaGraphInstantiate(&g->exec, graph, 0);
            } else {
                if (graph)
                    cudaGraphDestroy(graph);
                if (e2 != cudaSuccess)
                    e = e2;
            }
        }
        count_launch(l0 - launches_total());   // captured, not enqueued
    }
    if (origin)
        cudaStreamDestroy(origin);
    if (body)
        cudaStreamDestroy(body);
    if (rc == MG5_OK && e != cudaSuccess) {
        *err = std::string("graph solve: ") + cudaGetErrorString(e);
        rc = e == cudaErrorMemoryAllocation ? MG5_E_OOM : MG5_E_CUDA;
    }
    cudaGetLastError();
    if (rc != MG5_OK) {
        graph_free(g);
        return rc;
    }
    *out = g;
    return MG5_OK;
}

int graph_enqueue(GraphEntry *g, const double *delta, double *phi, double *grad, cudaStream_t st,
                  std::string *err)
{
    const size_t n3 = (size_t)g->N * g->N * g->N;
    cudaError_t e = cudaMemcpyAsync(g->delta, delta, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaGraphLaunch(g->exec, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(phi, g->phi, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, g->gout, 3 * n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&g->rb->ctl, g->ctl, sizeof(BoxCtl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&g->rb->cnt, g->cnt, sizeof(SolveCounters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&g->rb->ls0, g->ls, sizeof(LevelScal), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
        *err = std::string("graph solve: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return MG5_E_CUDA;
    }
    return MG5_OK;
}

void graph_checkin(GraphEntry *g) { g->busy = false; }

int graph_finish(GraphEntry *g, mg5_info *info)
{
    const BoxCtl &ctl = g->rb->ctl;
    const SolveCounters &cnt = g->rb->cnt;
    count_launch(g->stats.launches_fixed + g->stats.launches_per_iter * ctl.outer);
    int status = ctl.status;
    if (info) {
        info->status = status;
        info->outer_iters = g->hier ? ctl.outer : 0;
        info->cycles = ctl.outer * g->stats.inner;
        if (g->hierp) {
            info->levels = g->hierp->nlev;
            info->coarsest_n = g->hierp->q[info->levels - 1][0];
        } else {
            info->levels = g->hier ? g->hier->nlev : g->hier64->nlev;
            info->coarsest_n = g->hier ? g->hier->n[info->levels - 1] : g->hier64->n[info->levels - 1];
        }
        info->n_history = ctl.nhist;
        for (int k = 0; k < ctl.nhist && k < 64; ++k)
            info->history[k] = ctl.hist[k];
        info->rel_residual = ctl.rel;
        info->compat_c = g->rb->ls0.c;
        info->phi_mean_removed = g->rb->ls0.mean;
        const long long nc = info->coarsest_n;
        const long long coarse_cells =
            g->hierp ? (long long)int_cells(g->hierp->q[g->hierp->nlev - 1]) : nc * nc * nc;
        info->cell_updates = g->stats.cells_fixed + g->stats.cells_per_iter * ctl.outer +
                             (long long)cnt.coarse_sweeps * coarse_cells;
        info->coarse_sweeps = cnt.coarse_sweeps;
        info->disc_clamped = (long long)cnt.clamped;
    }
    if (status == MG5_OK && cnt.clamped > 0)
        status = MG5_W_DISC_CLAMP;
    g->busy = false;
    return status;
}

}  // namespace mg5

extern "C" {

// The FP64 solve from zero as one graph: f = s delta and ||f||, optional full-multigrid start,
// the first pre-smoothing and residual check, then the V-cycle as a WHILE node whose body is
// the coarse-grid correction, the post- and the next pre-smoothing and the check; the gauge and
// the force after it.  The body swaps every grid's buffers an even number of times (nu1 + nu2
// even), so the pointers it was captured with hold on every pass.
static int capture_fp64(mg5_ctx *ctx, GraphEntry *g, const mg5_params *p, cudaStream_t st,
                        cudaStream_t body_st)
{
    Hier *h = g->hier64;
    const int N = h->N;
    const long long n3 = (long long)N * N * N;
    Run64 R{ctx, h, p, st, {}, 0};
    R.lsb = g->ls;
    R.cntb = g->cnt;
    R.partb = g->partials;
    if (!R.bound() || !g->ctl || !g->phi || !g->delta) {
        ctx->err = "capture_fp64: entry scratch not allocated";
        return MG5_E_ARG;
    }
    for (int l = 0; l < h->nlev; ++l)
        R.hl[l] = p->h * (double)(1 << l);
    const long long L0 = launches_total();
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) {
        ctx->err = "capture_fp64: stream is not capturing";
        return MG5_E_ARG;
    }
    cudaGraphConditionalHandle hnd;
    CK(cudaGraphConditionalHandleCreate(&hnd, graph, 0, cudaGraphCondAssignDefault));
    CK(launch_ctl_init(g->ctl, p->tol, p->max_cycles, st));
    CK(cudaMemsetAsync(g->ls, 0, sizeof(LevelScal) * kScalSlots, st));
    CK(cudaMemsetAsync(g->cnt, 0, sizeof(SolveCounters), st));
    int nb = 0;
    CK(launch_scale(g->delta, p->s, h->f[0], n3, g->partials, &nb, st, 0.0, nullptr,
                    Fin{g->ls, FIN_FNORM, (double)n3}));
    CK(cudaMemsetAsync(g->phi, 0, n3 * sizeof(double), st));
    h->v[0] = g->phi;
    if (g->fmg)
        RET(R.fmg());
    for (int k = 0; k < p->nu1; ++k)
        RET(R.sweep(0));
    RET(R.resid_restrict(0));
    CK(launch_loop_check(g->ls, g->ctl, hnd, st));
    const long long cells_fixed = R.cu;
    // the WHILE node after everything captured so far
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    const long long L1 = launches_total();
    CK(cudaStreamBeginCaptureToGraph(body_st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    double *const v0_start = h->v[0];
    Run64 B = R;
    B.st = body_st;
    B.cu = 0;
    int rc = B.coarse_visit(1);
    if (rc == MG5_OK) {
        const cudaError_t e = launch_prolong_add<double>(h->v[1], h->v0[1], h->n[1], h->v[0], B.c(0),
                                                         B.c(1), body_st);
        rc = e == cudaSuccess ? MG5_OK : MG5_E_CUDA;
    }
    for (int k = 0; k < p->nu2 && rc == MG5_OK; ++k)
        rc = B.sweep(0);
    for (int k = 0; k < p->nu1 && rc == MG5_OK; ++k)
        rc = B.sweep(0);
    if (rc == MG5_OK)
        rc = B.resid_restrict(0);
    if (rc == MG5_OK && launch_loop_check(g->ls, g->ctl, hnd, body_st) != cudaSuccess)
        rc = MG5_E_CUDA;
    cudaGraph_t g_out = nullptr;
    const cudaError_t e_end = cudaStreamEndCapture(body_st, &g_out);
    RET(rc);
    CK(e_end);
    if (h->v[0] != v0_start) {
        ctx->err = "capture_fp64: the loop body does not return the grids to their buffers";
        return MG5_E_ARG;
    }
    const long long L2 = launches_total();
    // the iterate is in h->v[0]: bring it to the entry's phi, then the gauge and the force
    if (h->v[0] != g->phi)
        CK(cudaMemcpyAsync(g->phi, h->v[0], n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(launch_sum(g->phi, n3, g->partials, &nb, st, Fin{g->ls, FIN_MEAN, (double)n3}));
    CK(launch_sub_mean(g->phi, n3, &g->ls[0].mean, st));
    if (g->gout)
        CK(launch_force(g->phi, N, N, N, 0, p->h, 1, g->gout, st));
    g->stats.launches_fixed = (L1 - L0) + (launches_total() - L2);
    g->stats.launches_per_iter = L2 - L1;
    g->stats.cells_per_iter = B.cu;
    g->stats.cells_fixed = cells_fixed;
    g->stats.inner = 1;
    return MG5_OK;
}

// Build an FP64 entry: its own hierarchy, scalars and staging, the capture, the instantiation.
static int graph_build64(mg5_ctx *ctx, int N, const mg5_params *p, bool grad, bool fmg,
                         GraphEntry **out)
{
    *out = nullptr;
    GraphEntry *g = new GraphEntry();
    g->N = N;
    g->prm = *p;
    g->grad = grad;
    g->fmg = fmg;
    g->sched = schedule_version();   // read before the capture reads the schedules
    const size_t n3 = (size_t)N * N * N;
    cudaError_t e = alloc_hier_raw(N, &g->hier64);
    if (e == cudaSuccess)
        e = alloc_partials(&g->partials);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->ls, sizeof(LevelScal) * kScalSlots);
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->cnt, sizeof(SolveCounters));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->ctl, sizeof(BoxCtl));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->delta, n3 * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&g->phi, n3 * sizeof(double));
    if (e == cudaSuccess && grad)
        e = cudaMalloc((void **)&g->gout, 3 * n3 * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&g->rb, sizeof(GraphReadback));
    g->bytes = graph_entry_bytes64(N, grad);
    cudaStream_t origin = nullptr, body = nullptr;
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking);
    int rc = e == cudaSuccess ? MG5_OK : (e == cudaErrorMemoryAllocation ? MG5_E_OOM : MG5_E_CUDA);
    if (rc != MG5_OK)
        ctx->err = std::string("graph solve: ") + cudaGetErrorString(e);
    const long long l0 = launches_total();
    const bool prof_on = ctx->prof.on;
    if (rc == MG5_OK) {
        ctx->prof.on = false;
        e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = capture_fp64(ctx, g, p, origin, body);
            cudaGraph_t graph = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
            if (rc == MG5_OK && e2 == cudaSuccess) {
                g->graph = graph;
                e = cudaGraphInstantiate(&g->exec, graph, 0);
            } else {
                if (graph)
                    cudaGraphDestroy(graph);
                if (e2 != cudaSuccess)
                    e = e2;
            }
        }
        ctx->prof.on = prof_on;
        count_launch(l0 - launches_total());   // captured, not enqueued
        if (rc == MG5_OK && e != cudaSuccess) {
            ctx->err = std::string("graph solve: ") + cudaGetErrorString(e);
            rc = MG5_E_CUDA;
        }
    }
    if (origin)
        cudaStreamDestroy(origin);
    if (body)
        cudaStreamDestroy(body);
    cudaGetLastError();
    if (rc != MG5_OK) {
        graph_free(g);
        return rc;
    }
    *out = g;
    return MG5_OK;
}

// The cached graph for (N, params, grad), or a new capture (evicting the least
// recently used entries while the cache is full or the budget would be exceeded).
static int get_graph_entry(mg5_ctx *ctx, int N, const mg5_params *p, bool grad, bool fmg,
                           GraphEntry **out)
{
    // entries captured under an older schedule table are not replayed again: free them (every
    // entry is idle here, this context's solves have synchronised)
    for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
        GraphEntry *g = *it;
        if (!g->busy && !g->current()) {
            it = ctx->graphs.erase(it);
            ctx->held -= g->bytes;
            graph_free(g);
        } else {
            ++it;
        }
    }
    for (GraphEntry *g : ctx->graphs)
        if (!g->busy && g->N == N && g->grad == grad && g->fmg == fmg && same_params(g->prm, *p) &&
            g->current()) {
            g->busy = true;
            g->last_use = ++ctx->graph_clock;
            *out = g;
            return MG5_OK;
        }
    const bool fp64 = p->precision == MG5_FP64;
    const size_t need = fp64 ? graph_entry_bytes64(N, grad) : graph_entry_bytes(N, grad);
    while (ctx->graphs.size() >= kGraphCacheMax || (ctx->budget && ctx->held + need > ctx->budget)) {
        GraphEntry *v = graph_take_idle(ctx);   // every entry is idle: this context's solves have synchronised
        if (!v)
            break;
        graph_free(v);
    }
    if (ctx->budget && ctx->held + need > ctx->budget) {
        ctx->err = "graph solve would exceed the context's HBM budget";
        return MG5_E_OOM;
    }
    GraphEntry *g = nullptr;
    int rc;
    if (fp64) {
        rc = graph_build64(ctx, N, p, grad, fmg, &g);
    } else {
        const bool prof_on = ctx->prof.on;
        ctx->prof.on = false;
        rc = graph_build(ctx->device, N, p, grad, &g, &ctx->err);
        ctx->prof.on = prof_on;
    }
    RET(rc);
    graph_insert(ctx, g);
    *out = g;
    return MG5_OK;
}

}  // extern "C"

namespace mg5 {

bool graph_capturable(int N, const mg5_params *p)
{
    if (p->precision != MG5_FP64)
        return true;
    int sz[kMaxLevels];
    return num_levels(N, sz) >= 2 && (p->nu1 + p->nu2) % 2 == 0;
}

int graph_build_in(mg5_ctx *ctx, int N, const mg5_params *p, bool grad, GraphEntry **out,
                   std::string *err)
{
    if (p->precision != MG5_FP64)
        return graph_build(ctx->device, N, p, grad, out, err);
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        *err = "graph solve: cannot select the device";
        return MG5_E_CUDA;
    }
    const int rc = graph_build64(ctx, N, p, grad, false, out);
    if (rc != MG5_OK)
        *err = ctx->err;
    return rc;
}

}  // namespace mg5

extern "C" {

// A solve from zero through the cached graph: copy in, one graph launch, copy out.
static int solve_graph(mg5_ctx *ctx, const double *delta, int N, const mg5_params *p, double *phi,
                       double *grad, bool fmg, mg5_info *info, cudaStream_t st)
{
    GraphEntry *g = nullptr;
    RET(get_graph_entry(ctx, N, p, grad != nullptr, fmg, &g));
    int rc = graph_enqueue(g, delta, phi, grad, st, &ctx->err);
    if (rc == MG5_OK && ctx_wait(ctx, st) != cudaSuccess) {
        ctx->err = std::string("graph solve: ") + cudaGetErrorString(cudaGetLastError());
        rc = MG5_E_CUDA;
    }
    if (rc != MG5_OK) {
        graph_checkin(g);
        return rc;
    }
    return graph_finish(g, info);
}

static bool batch_matches(const BatchSet *b, int nbox, const double *const *delta, const int *N,
                          const mg5_params *p, double *const *phi, double *const *grad)
{
    if (!b || b->nbox != nbox || b->sched != schedule_version())
        return false;
    for (int i = 0; i < nbox; ++i)
        if (b->N[i] != N[i] || !same_params(b->prm[i], p[i]) || b->delta[i] != delta[i] ||
            b->phi[i] != phi[i] || b->grad[i] != (grad ? grad[i] : nullptr))
            return false;
    return true;
}

static int build_batch(mg5_ctx *ctx, int nbox, const double *const *delta, const int *N,
                       const mg5_params *p, double *const *phi, double *const *grad)
{
    free_batch(ctx);
    BatchSet *b = new BatchSet();
    ctx->batch = b;
    b->sched = schedule_version();   // read before the capture reads the schedules
    b->nbox = nbox;
    b->N.assign(N, N + nbox);
    b->prm.assign(p, p + nbox);
    b->delta.assign(delta, delta + nbox);
    b->phi.assign(phi, phi + nbox);
    b->grad.resize(nbox);
    for (int i = 0; i < nbox; ++i)
        b->grad[i] = grad ? grad[i] : nullptr;
    const size_t per_box = sizeof(double2) * kMaxPartials + sizeof(LevelScal) * kScalSlots +
                           sizeof(SolveCounters);
    b->bytes = per_box * nbox + sizeof(BoxCtl) * nbox;
    if (ctx->budget && ctx->held + b->bytes > ctx->budget) {
        ctx->err = "batch scratch would exceed the context's HBM budget";
        free_batch(ctx);
        return MG5_E_OOM;
    }
    ctx->held += b->bytes;
    b->hier.assign(nbox, nullptr);
    b->partials.assign(nbox, nullptr);
    b->ls.assign(nbox, nullptr);
    b->cnt.assign(nbox, nullptr);
    b->stats.assign(nbox, CaptureStats{});
    CK(cudaMalloc((void **)&b->ctl, sizeof(BoxCtl) * nbox));
    for (int i = 0; i < nbox; ++i) {
        int rc = alloc_mixed(N[i], ctx->budget, &ctx->held, &b->hier[i], &ctx->err);
        if (rc != MG5_OK) {
            free_batch(ctx);
            return rc;
        }
        CK(alloc_partials(&b->partials[i]));
        CK(cudaMalloc((void **)&b->ls[i], sizeof(LevelScal) * kScalSlots));
        CK(cudaMalloc((void **)&b->cnt[i], sizeof(SolveCounters)));
    }
    // capture: fork one branch per box off a private origin stream
    cudaStream_t origin = nullptr, body = nullptr;
    std::vector<cudaStream_t> br(nbox, nullptr);
    std::vector<cudaEvent_t> join(nbox, nullptr);
    cudaEvent_t fork = nullptr;
    auto cleanup = [&]() {
        for (cudaEvent_t e : join)
            if (e)
                cudaEventDestroy(e);
        for (cudaStream_t q : br)
            if (q)
                cudaStreamDestroy(q);
        if (fork)
            cudaEventDestroy(fork);
        if (body)
            cudaStreamDestroy(body);
        if (origin)
            cudaStreamDestroy(origin);
    };
    const bool prof_on = ctx->prof.on;
    ctx->prof.on = false;   // event records are not allowed inside loop bodies
    const long long launches_before = launches_total();
    int rc = MG5_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithFlags(&body, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < nbox && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess)
        e = cudaEventRecord(fork, origin);
    for (int i = 0; i < nbox && e == cudaSuccess && rc == MG5_OK; ++i) {
        e = cudaStreamWaitEvent(br[i], fork, 0);
        if (e != cudaSuccess)
            break;
        MixedShared sh{b->partials[i], b->ls[i], b->cnt[i], ctx->h_rel, nullptr};
        rc = capture_mixed(b->hier[i], sh, delta[i], &p[i], phi[i], b->grad[i], b->ctl + i, br[i],
                           body, &b->stats[i], &ctx->err);
        if (rc == MG5_OK) {
            e = cudaEventRecord(join[i], br[i]);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(origin, join[i], 0);
        }
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(origin, &g);
    if (e == cudaSuccess)
        e = e2;
    ctx->prof.on = prof_on;
    count_launch(launches_before - launches_total());   // captured, not enqueued
    if (rc == MG5_OK && e == cudaSuccess) {
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
    } else if (g) {
        cudaGraphDestroy(g);
    }
    cleanup();
    if (rc != MG5_OK) {
        free_batch(ctx);
        return rc;
    }
    if (e != cudaSuccess) {
        ctx->err = std::string("batch graph: ") + cudaGetErrorString(e);
        cudaGetLastError();
        free_batch(ctx);
        return MG5_E_CUDA;
    }
    return MG5_OK;
}

int mg5_solve_batch(mg5_ctx *ctx, int nbox, const double *const *delta, const int *N,
                    const mg5_params *p, double *const *phi, double *const *grad, mg5_info *info,
                    void *stream)
{
    if (!ctx || nbox < 1 || !delta || !N || !p || !phi)
        return MG5_E_ARG;
    bool all_mixed = true;
    for (int i = 0; i < nbox; ++i) {
        if (!delta[i] || !phi[i])
            return MG5_E_ARG;
        RET(check_size(N[i]));
        RET(check_params(&p[i]));
        all_mixed = all_mixed && p[i].precision == MG5_MIXED;
    }
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    if (info)
        std::memset(info, 0, sizeof(mg5_info) * nbox);
    if (!all_mixed) {
        // FP64 boxes: one host-driven solve after the other on the caller's stream
        int worst = MG5_OK;
        for (int i = 0; i < nbox; ++i) {
            int rc = mg5_solve_fifth_force(ctx, delta[i], N[i], &p[i], 0, phi[i],
                                           grad ? grad[i] : nullptr, info ? info + i : nullptr,
                                           stream);
            if (rc == MG5_E_CUDA || rc == MG5_E_ARG || rc == MG5_E_OOM)
                return rc;
            if (rc < 0 || (worst == MG5_OK && rc > 0))
                worst = rc;
        }
        return worst;
    }
    if (!batch_matches(ctx->batch, nbox, delta, N, p, phi, grad)) {
        if (ctx->autotune)
            for (int i = 0; i < nbox; ++i)
                RET(ctx_autotune(ctx, N[i], MG5_MIXED, st));
        RET(build_batch(ctx, nbox, delta, N, p, phi, grad));
    }
    BatchSet *b = ctx->batch;
    CK(cudaEventRecord(ctx->ev0, st));
    CK(cudaGraphLaunch(b->exec, st));
    CK(cudaEventRecord(ctx->ev1, st));
    std::vector<BoxCtl> ctl(nbox);
    CK(cudaMemcpyAsync(ctl.data(), b->ctl, sizeof(BoxCtl) * nbox, cudaMemcpyDeviceToHost, st));
    std::vector<SolveCounters> cnt(nbox);
    std::vector<LevelScal> ls0(nbox);
    for (int i = 0; i < nbox; ++i) {
        CK(cudaMemcpyAsync(&cnt[i], b->cnt[i], sizeof(SolveCounters), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&ls0[i], b->ls[i], sizeof(LevelScal), cudaMemcpyDeviceToHost, st));
    }
    CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    int worst = MG5_OK;
    for (int i = 0; i < nbox; ++i) {
        const CaptureStats &cs = b->stats[i];
        count_launch(cs.launches_fixed + cs.launches_per_iter * ctl[i].outer);
        int status = ctl[i].status;
        if (status == MG5_OK && cnt[i].clamped > 0)
            status = MG5_W_DISC_CLAMP;
        if (status < 0 || (worst == MG5_OK && status > 0))
            worst = status;
        if (info) {
            mg5_info &o = info[i];
            o.status = status;
            o.outer_iters = ctl[i].outer;
            o.cycles = ctl[i].outer * cs.inner;
            o.levels = b->hier[i]->nlev;
            o.coarsest_n = b->hier[i]->n[o.levels - 1];
            o.n_history = ctl[i].nhist;
            for (int k = 0; k < ctl[i].nhist && k < 64; ++k)
                o.history[k] = ctl[i].hist[k];
            o.rel_residual = ctl[i].rel;
            o.compat_c = ls0[i].c;
            o.phi_mean_removed = ls0[i].mean;
            o.disc_clamped = (long long)cnt[i].clamped;
            const long long nc = o.coarsest_n;
            o.cell_updates = cs.cells_per_iter * ctl[i].outer + (long long)cnt[i].coarse_sweeps * nc * nc * nc;
            o.coarse_sweeps = cnt[i].coarse_sweeps;
            o.ms_total = ms;
        }
    }
    return worst;
}

int mg5_step_sweep(mg5_ctx *ctx, const double *in, double *out, const double *f, double c, int N,
                   double h, double alpha, void *stream)
{
    if (!ctx || !in || !out || !f || in == out || N < 2 || (N & 1) || !(h > 0.0))
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    double *cd = &ctx->ls[kStepSlot].c;
    CK(cudaMemcpyAsync(cd, &c, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(launch_sweep<double>(in, out, f, cd, N, make_coef<double>(h, alpha), &ctx->cnt->clamped, st));
    CK(cudaStreamSynchronize(st));
    return MG5_OK;
}

int mg5_step_sweep_f32(mg5_ctx *ctx, const float *in, float *out, const float *f, const float *B,
                       double c, int N, double h, double alpha, int variant, void *stream)
{
    if (!ctx || !in || !out || !f || in == out || N < 2 || (N & 1) || !(h > 0.0) ||
        variant < 0 || variant > 2 || (variant == 2 && (!B || !march_ok(N))))
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    double *cd = &ctx->ls[kStepSlot].c;
    CK(cudaMemcpyAsync(cd, &c, sizeof(double), cudaMemcpyHostToDevice, st));
    const CoefT<float> cf = make_coef<float>(h, alpha);
    if (variant == 2)
        CK(launch_sweep_march(in, out, f, B, cd, N, cf, &ctx->cnt->clamped, st));
    else if (variant == 1)
        CK(launch_sweep_fused<float>(in, out, f, cd, N, cf, &ctx->cnt->clamped, st, B));
    else
        CK(launch_sweep<float>(in, out, f, cd, N, cf, &ctx->cnt->clamped, st, B));
    CK(cudaStreamSynchronize(st));
    return MG5_OK;
}

int mg5_step_resid_restrict_f32(mg5_ctx *ctx, const float *e, const float *f, const float *B,
                                double c, int N, double h, double alpha, int variant, float *ec,
                                float *rc, double *stats, void *stream)
{
    if (!ctx || !e || !f || !B || !ec || !rc || N < 2 || (N & 1) || !(h > 0.0) || variant < 0 ||
        variant > 1 || (variant == 1 && !resid_march_ok(N)))
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    LevelScal *ls = ctx->ls + kStepSlot;
    CK(cudaMemsetAsync(ls, 0, sizeof(LevelScal), st));
    CK(cudaMemcpyAsync(&ls->c, &c, sizeof(double), cudaMemcpyHostToDevice, st));
    const CoefT<float> cf = make_coef<float>(h, alpha);
    const Fin fin{ls, FIN_STATS, (double)N * N * N};
    int nb = 0;
    if (variant == 1)
        CK(launch_resid_restrict_march(e, f, &ls->c, N, cf, ec, ec, rc, ctx->partials, &nb, st, B,
                                       fin));
    else
        CK(launch_resid_restrict<float>(e, f, &ls->c, N, cf, ec, ec, rc, ctx->partials, &nb, st, B,
                                        fin));
    LevelScal out;
    CK(cudaMemcpyAsync(&out, ls, sizeof(LevelScal), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (stats) {
        stats[0] = out.m;
        stats[1] = out.rnorm;
    }
    return MG5_OK;
}

int mg5_step_sweep_fused(mg5_ctx *ctx, const double *in, double *out, const double *f, double c,
                         int N, double h, double alpha, void *stream)
{
    if (!ctx || !in || !out || !f || in == out || N < 2 || (N & 1) || !(h > 0.0))
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    double *cd = &ctx->ls[kStepSlot].c;
    CK(cudaMemcpyAsync(cd, &c, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(launch_sweep_fused<double>(in, out, f, cd, N, make_coef<double>(h, alpha), &ctx->cnt->clamped,
                                  st));
    CK(cudaStreamSynchronize(st));
    return MG5_OK;
}

int mg5_step_operator(mg5_ctx *ctx, const double *phi, int N, double h, double alpha, double *out,
                      void *stream)
{
    if (!ctx || !phi || !out || N < 1 || !(h > 0.0))
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(launch_operator<double>(phi, N, make_coef<double>(h, alpha), out, (cudaStream_t)stream));
    return MG5_OK;
}

int mg5_step_residual(mg5_ctx *ctx, const double *phi, const double *f, double c, int N, double h,
                      double alpha, double *r, void *stream)
{
    if (!ctx || !phi || !f || !r || N < 1 || !(h > 0.0))
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    double *cd = &ctx->ls[kStepSlot].c;
    CK(cudaMemcpyAsync(cd, &c, sizeof(double), cudaMemcpyHostToDevice, st));
    int nb = 0;
    CK(launch_residual<double>(phi, f, cd, N, make_coef<double>(h, alpha), r, ctx->partials, &nb, st));
    CK(cudaStreamSynchronize(st));
    return MG5_OK;
}

int mg5_step_restrict(mg5_ctx *ctx, const double *fine, int N, double *coarse, void *stream)
{
    if (!ctx || !fine || !coarse || N < 2 || (N & 1))
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(launch_restrict<double>(fine, N, coarse, (cudaStream_t)stream));
    return MG5_OK;
}

int mg5_step_prolong_add(mg5_ctx *ctx, const double *coarse, int Nc, double *fine, void *stream)
{
    if (!ctx || !coarse || !fine || Nc < 1)
        return MG5_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(launch_prolong_add<double>(coarse, nullptr, Nc, fine, nullptr, nullptr, (cudaStream_t)stream));
    return MG5_OK;
}

}  // extern "C"
