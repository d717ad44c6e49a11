// mg5_mixed.cu -- mixed-precision solve: FP64 residual + defect correction
// around FP32 FAS V-cycles on the correction equation (the FP32 kernels take
// the correction form of the cell arithmetic, see mg5_dev.cuh).
//
// Outer step k:  r = s delta + c - op(phi) in FP64 (its mean m is projected
// out; ||r - m|| / ||s delta|| is the stopping test), B = fp32(phi) restricted
// to every grid, then `inner_cycles` FP32 V-cycles for
//     op(B + e) - op(B) = r - m + c_e,   e = 0 at the start,
// then phi += e and c += c_e in FP64.  Because only the residual and the
// update are formed in FP64, the FP32 solve may stop at its own precision.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "mg5_fin.cuh"
#include "mg5_mixed.cuh"

namespace mg5 {

namespace {

constexpr double kCoarseRtol = 1e-3;

int levels_of(int N, int *sz)
{
    int L = 0, n = N;
    sz[L++] = n;
    while ((n / 2) % 2 == 0 && n / 2 >= 4 && L < kMixMaxLevels) {
        n /= 2;
        sz[L++] = n;
    }
    return L;
}

// r32 = fp32(f + c - op(phi)) and B = fp32(phi), FP64 arithmetic; partial sums of r.
// ZERO: phi = 0 (a solve from zero), where op(0) = 0 exactly: r = f + c without the
// stencil (the same values; a memory-bound pass instead of an FP64-bound one).
template <bool ZERO>
__global__ void k_resid64_mixed(const double *__restrict__ phi, const double *__restrict__ f,
                                const double *__restrict__ cptr, int n, CoefT<double> cf,
                                float *__restrict__ r32, float *__restrict__ B,
                                Moments *__restrict__ partials, Fin fin)
{
    const long long total = (long long)n * n * n;
    const double c = MG5_AT(cptr, 0);
    MomAcc<double> acc;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        if constexpr (ZERO) {
            const double res = MG5_AT(f, t) + c;
            MG5_AT(r32, t) = f64_to_f32_rn(res);
            MG5_AT(B, t) = 0.0f;
            acc.add(res);
            continue;
        }
        const int k = (int)(t % n);
        const long long q = t / n;
        const int j = (int)(q % n), i = (int)(q / n);
        const Rows r = periodic_rows(n, i, j);
        const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
        St<double> s;
        gather(phi, phi, r, k, kp, km, s);
        const double res = cell_residual(s, MG5_AT(f, t) + c, cf);
        MG5_AT(r32, t) = f64_to_f32_rn(res);
        MG5_AT(B, t) = f64_to_f32_rn(s.c);
        acc.add(res);
    }
    const Moments m = block_moments(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = m;
    finalize_if_last(reinterpret_cast<double2 *>(partials), fin);
}

__global__ void k_update_mixed(double *__restrict__ phi, const float *__restrict__ e, long long n3)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n3)
        MG5_AT(phi, t) += f32_to_f64(MG5_AT(e, t));
}

// scalar bookkeeping: 0: a.c -= a.m ; 1: b.c = -a.m ; 2: a.c += b.c
__global__ void k_scal(LevelScal *a, LevelScal *b, int op)
{
    a = &MG5_AT(a, 0);
    b = &MG5_AT(b, 0);
    if (op == 0)
        a->c -= a->m;
    else if (op == 1)
        b->c = -a->m;
    else
        a->c += b->c;
}

struct RunMix {
    MixedHier *h;
    const MixedShared &sh;
    const mg5_params *p;
    cudaStream_t st;
    std::string *err;
    double hl[kMixMaxLevels];
    long long cu = 0;  // cell updates of the non-coarsest sweeps

    LevelScal *ls(int l) { return sh.ls + kInnerBase + l; }
    double *c(int l) { return &ls(l)->c; }
    double *m(int l) { return &ls(l)->m; }

    int fail(const char *what, cudaError_t e)
    {
        *err = std::string(what) + ": " + cudaGetErrorString(e);
        return MG5_E_CUDA;
    }

    int sweep(int l)
    {
        ProfScope ps(sh.prof, l == 0 ? PK_SWEEP32 : PK_SWEEP32C, st, (double)(h->n[l]) * (h->n[l]) * (h->n[l]));
        const CoefT<float> cf = make_coef<float>(hl[l], p->alpha, omega_of(p));
        int dev = 0;
        cudaGetDevice(&dev);
        cudaError_t e = launch_sweep_sched<float>(sweep_schedule(dev, MG5_MIXED, h->n[l]), h->e[l],
                                                  h->etmp[l], h->f[l], c(l), h->n[l], cf,
                                                  &sh.cnt->clamped, st, h->B[l]);
        if (e != cudaSuccess)
            return fail("sweep32", e);
        std::swap(h->e[l], h->etmp[l]);
        cu += (long long)h->n[l] * h->n[l] * h->n[l];
        return MG5_OK;
    }

    int coarsest(int l)
    {
        ProfScope ps(sh.prof, PK_COARSEST32, st);
        if (h->spec[0] && h->n[l] >= kSpectralMinSide) {
            const cudaError_t e = launch_coarsest_spectral<float>(
                h->e[l], h->etmp[l], h->f[l], h->n[l], make_coef<float>(hl[l], p->alpha, omega_of(p)),
                ls(l), kSpectralIters, &sh.cnt->clamped, &sh.cnt->coarse_sweeps, sh.partials,
                h->spec[0], h->spec[1], st, h->B[l]);
            return e == cudaSuccess ? MG5_OK : fail("coarsest32", e);
        }
        cudaError_t e = launch_coarsest<float>(h->e[l], h->etmp[l], h->f[l], h->n[l],
                                               make_coef<float>(hl[l], p->alpha, omega_of(p)), c(l),
                                               p->nu_coarse, kCoarseRtol, &sh.cnt->clamped,
                                               &sh.cnt->coarse_sweeps, st, h->B[l]);
        return e == cudaSuccess ? MG5_OK : fail("coarsest32", e);
    }

    int resid_restrict(int l)
    {
        int nb = 0;
        ProfScope ps(sh.prof, PK_RESTRICT32, st, (double)(h->n[l]) * (h->n[l]) * (h->n[l]));
        const double n3 = (double)h->n[l] * h->n[l] * h->n[l];
        const CoefT<float> cf = make_coef<float>(hl[l], p->alpha);
        const Fin fin{ls(l), FIN_RESID, n3};
        cudaError_t e =
            resid_march_ok(h->n[l])
                ? launch_resid_restrict_march(h->e[l], h->f[l], c(l), h->n[l], cf, h->e[l + 1],
                                              h->e0[l + 1], h->f[l + 1], sh.partials, &nb, st,
                                              h->B[l], fin)
                : launch_resid_restrict<float>(h->e[l], h->f[l], c(l), h->n[l], cf, h->e[l + 1],
                                               h->e0[l + 1], h->f[l + 1], sh.partials, &nb, st,
                                               h->B[l], fin);
        return e == cudaSuccess ? MG5_OK : fail("resid_restrict32", e);
    }

    int coarse_visit(int l)
    {
        cudaError_t e;
        if (l == h->nlev - 2 && bottom_ok(h->n[l]) && h->n[l + 1] < kSpectralMinSide) {
            // this grid and the coarsest one in a single launch (k_bottom.cu)
            ProfScope ps(sh.prof, PK_COARSEST32, st);
            e = launch_bottom<float>(h->e[l], h->f[l], h->B[l], h->B[l + 1], h->n[l],
                                     make_coef<float>(hl[l], p->alpha, omega_of(p)),
                                     make_coef<float>(hl[l + 1], p->alpha, omega_of(p)), ls(l - 1),
                                     ls(l), ls(l + 1), p->nu1, p->nu2, p->nu_coarse, kCoarseRtol,
                                     &sh.cnt->clamped, &sh.cnt->coarse_sweeps, st);
            if (e != cudaSuccess)
                return fail("bottom32", e);
            cu += (long long)(p->nu1 + p->nu2) * h->n[l] * h->n[l] * h->n[l];
            return MG5_OK;
        }
        {
            ProfScope ps(sh.prof, PK_COARSE_RHS32, st, (double)(h->n[l]) * (h->n[l]) * (h->n[l]));
            e = launch_coarse_rhs<float>(h->e[l], h->f[l], m(l - 1), c(l), h->n[l],
                                         make_coef<float>(hl[l], p->alpha), st, h->B[l]);
        }
        if (e != cudaSuccess)
            return fail("coarse_rhs32", e);
        if (l == h->nlev - 1)
            return coarsest(l);
        for (int s = 0; s < p->nu1; ++s)
            if (int rc = sweep(l))
                return rc;
        if (int rc = resid_restrict(l))
            return rc;
        if (int rc = coarse_visit(l + 1))
            return rc;
        {
            ProfScope ps(sh.prof, PK_PROLONG32, st, (double)(h->n[l]) * (h->n[l]) * (h->n[l]));
            e = launch_prolong_add<float>(h->e[l + 1], h->e0[l + 1], h->n[l + 1], h->e[l], c(l),
                                          c(l + 1), st);
        }
        if (e != cudaSuccess)
            return fail("prolong32", e);
        for (int s = 0; s < p->nu2; ++s)
            if (int rc = sweep(l))
                return rc;
        return MG5_OK;
    }

    // one inner V-cycle on the finest grid
    int vcycle0()
    {
        if (h->nlev == 1)
            return coarsest(0);
        for (int s = 0; s < p->nu1; ++s)
            if (int rc = sweep(0))
                return rc;
        if (int rc = resid_restrict(0))
            return rc;
        if (int rc = coarse_visit(1))
            return rc;
        cudaError_t e;
        {
            ProfScope ps(sh.prof, PK_PROLONG32, st, (double)(h->n[0]) * (h->n[0]) * (h->n[0]));
            e = launch_prolong_add<float>(h->e[1], h->e0[1], h->n[1], h->e[0], c(0), c(1), st);
        }
        if (e != cudaSuccess)
            return fail("prolong32", e);
        for (int s = 0; s < p->nu2; ++s)
            if (int rc = sweep(0))
                return rc;
        return MG5_OK;
    }
};

}  // namespace

size_t mixed_bytes(int N)
{
    int sz[kMixMaxLevels];
    const int L = levels_of(N, sz);
    const size_t n3 = (size_t)N * N * N;
    size_t b = n3 * sizeof(double) + 4 * n3 * sizeof(float);
    for (int l = 1; l < L; ++l)
        b += 5 * (size_t)sz[l] * sz[l] * sz[l] * sizeof(float);
    if (L > 1 && sz[L - 1] >= kSpectralMinSide)
        b += 2 * (size_t)sz[L - 1] * sz[L - 1] * sz[L - 1] * sizeof(float2);
    return b;
}

void free_mixed(MixedHier *m, size_t *held)
{
    if (!m)
        return;
    auto fr = [&](void *p) {
        if (p)
            cudaFree(p);
    };
    fr(m->f64);
    for (int l = 0; l < m->nlev; ++l) {
        fr(m->B[l]);
        fr(m->e[l]);
        fr(m->etmp[l]);
        fr(m->f[l]);
        fr(m->e0[l]);
    }
    fr(m->spec[0]);
    fr(m->spec[1]);
    *held -= m->bytes;
    delete m;
}

int alloc_mixed(int N, size_t budget, size_t *held, MixedHier **out, std::string *err)
{
    const size_t need = mixed_bytes(N);
    if (budget && *held + need > budget) {
        *err = "scratch would exceed the context's HBM budget";
        return MG5_E_OOM;
    }
    MixedHier *m = new MixedHier();
    m->N = N;
    m->nlev = levels_of(N, m->n);
    m->bytes = need;
    *held += need;
    cudaError_t e = cudaMalloc((void **)&m->f64, (size_t)N * N * N * sizeof(double));
    for (int l = 0; l < m->nlev && e == cudaSuccess; ++l) {
        const size_t b = (size_t)m->n[l] * m->n[l] * m->n[l] * sizeof(float);
        e = cudaMalloc((void **)&m->B[l], b);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&m->e[l], b);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&m->etmp[l], b);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&m->f[l], b);
        if (e == cudaSuccess && l > 0)
            e = cudaMalloc((void **)&m->e0[l], b);
    }
    const int nc = m->n[m->nlev - 1];
    if (e == cudaSuccess && m->nlev > 1 && nc >= kSpectralMinSide)
        for (float2 **q : {&m->spec[0], &m->spec[1]})
            if (e == cudaSuccess)
                e = cudaMalloc((void **)q, (size_t)nc * nc * nc * sizeof(float2));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        free_mixed(m, held);
        return e == cudaErrorMemoryAllocation ? MG5_E_OOM : MG5_E_CUDA;
    }
    *out = m;
    return MG5_OK;
}

// ---------------------------------------------------------------- phases

#define CKM(call)                                                           \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) {                                            \
            *err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
            return MG5_E_CUDA;                                              \
        }                                                                   \
    } while (0)

namespace {

// f64 = s delta, ||f64||, scalars and counters cleared
int phase_setup(MixedHier *h, const MixedShared &sh, const double *delta, const mg5_params *p,
                cudaStream_t st, std::string *err)
{
    const long long n3 = (long long)h->N * h->N * h->N;
    CKM(cudaMemsetAsync(sh.ls, 0, sizeof(LevelScal) * kScalSlots, st));
    CKM(cudaMemsetAsync(sh.cnt, 0, sizeof(SolveCounters), st));
    int nb = 0;
    CKM(launch_scale(delta, p->s, h->f64, n3, sh.partials, &nb, st, 0.0, nullptr,
                     Fin{sh.ls, FIN_FNORM, (double)n3}));
    return MG5_OK;
}

// r32 = fp32(s delta + c - op(phi)) and B = fp32(phi) in FP64 arithmetic; stats of r
int phase_residual(MixedHier *h, const MixedShared &sh, const mg5_params *p, double *phi,
                   cudaStream_t st, std::string *err, bool zero = false)
{
    const int N = h->N;
    const long long n3 = (long long)N * N * N;
    const int cap = zero ? kReduceBlocks : kReduceBlocksFp64;   // ZERO: memory-bound
    int grid = blocks_for(n3);
    if (grid > cap)
        grid = cap;
    {
        ProfScope ps(sh.prof, PK_RESID64_MIXED, st, (double)n3);
        const CoefT<double> cf = make_coef<double>(p->h, p->alpha);
        Moments *mp = reinterpret_cast<Moments *>(sh.partials);
        const Fin fin{sh.ls, FIN_STATS, (double)n3};
        if (zero)
            k_resid64_mixed<true><<<grid, kBlock, 0, st>>>(phi, h->f64, &sh.ls[0].c, N, cf,
                                                           h->f[0], h->B[0], mp, fin);
        else
            k_resid64_mixed<false><<<grid, kBlock, 0, st>>>(phi, h->f64, &sh.ls[0].c, N, cf,
                                                            h->f[0], h->B[0], mp, fin);
    }
    count_launch(1);
    CKM(cudaGetLastError());
    return MG5_OK;
}

// restrict the base, `inner` FP32 V-cycles on the correction, phi += e, c += c_e
int phase_work(RunMix &R, double *phi, int inner, std::string *err)
{
    MixedHier *h = R.h;
    const MixedShared &sh = R.sh;
    cudaStream_t st = R.st;
    const long long n3 = (long long)h->N * h->N * h->N;
    for (int l = 1; l < h->nlev; ++l)
        CKM(launch_restrict<float>(h->B[l - 1], h->n[l - 1], h->B[l], st));
    CKM(cudaMemsetAsync(h->e[0], 0, n3 * sizeof(float), st));
    k_scal<<<1, 1, 0, st>>>(sh.ls, R.ls(0), 1);  // inner c = -m
    count_launch(1);
    CKM(cudaGetLastError());
    for (int it = 0; it < inner; ++it)
        if (int rc = R.vcycle0())
            return rc;
    {
        ProfScope ps(sh.prof, PK_UPDATE_MIXED, st, (double)n3);
        k_update_mixed<<<blocks_for(n3), kBlock, 0, st>>>(phi, h->e[0], n3);
    }
    count_launch(1);
    CKM(cudaGetLastError());
    k_scal<<<1, 1, 0, st>>>(sh.ls, R.ls(0), 2);  // c += c_e
    count_launch(1);
    CKM(cudaGetLastError());
    return MG5_OK;
}

// report the projected c, gauge phi to mean zero
int phase_finish(MixedHier *h, const MixedShared &sh, double *phi, cudaStream_t st, std::string *err)
{
    const long long n3 = (long long)h->N * h->N * h->N;
    k_scal<<<1, 1, 0, st>>>(sh.ls, sh.ls, 0);
    count_launch(1);
    CKM(cudaGetLastError());
    int nb = 0;
    CKM(launch_sum(phi, n3, sh.partials, &nb, st, Fin{sh.ls, FIN_MEAN, (double)n3}));
    CKM(launch_sub_mean(phi, n3, &sh.ls[0].mean, st));
    return MG5_OK;
}

}  // namespace

int solve_mixed(MixedHier *h, const MixedShared &sh, const double *delta, const mg5_params *p,
                double *phi, mg5_info *info, cudaStream_t st, std::string *err, bool zero_start)
{
    RunMix R{h, sh, p, st, err, {}, 0};
    for (int l = 0; l < h->nlev; ++l)
        R.hl[l] = p->h * (double)(1 << l);
    const int inner = inner_cycles_for(p);
    if (int rc = phase_setup(h, sh, delta, p, st, err))
        return rc;
    int status = MG5_E_NOT_CONVERGED;
    double best = INFINITY;
    int outer = 0;
    for (;; ++outer) {
        if (int rc = phase_residual(h, sh, p, phi, st, err, zero_start && outer == 0))
            return rc;
        CKM(cudaMemcpyAsync(sh.h_rel, &sh.ls[0].rel, sizeof(double), cudaMemcpyDeviceToHost, st));
        CKM(host_wait(st, sh.wait_ev));
        const double rel = *sh.h_rel;
        if (info) {
            if (outer < 64) {
                info->history[outer] = rel;
                info->n_history = outer + 1;
            }
            info->rel_residual = rel;
        }
        if (!std::isfinite(rel)) {
            status = MG5_E_NONFINITE;
            break;
        }
        if (rel <= p->tol) {
            status = MG5_OK;
            break;
        }
        best = std::min(best, rel);
        if (outer >= 3 && rel > 10.0 * best) {
            status = MG5_E_DIVERGED;
            break;
        }
        if (outer >= p->max_cycles) {
            status = MG5_E_NOT_CONVERGED;
            break;
        }
        if (int rc = phase_work(R, phi, inner, err))
            return rc;
    }
    if (int rc = phase_finish(h, sh, phi, st, err))
        return rc;
    if (info) {
        info->cycles = outer * inner;
        info->outer_iters = outer;
        info->levels = h->nlev;
        info->coarsest_n = h->n[h->nlev - 1];
        info->cell_updates = R.cu;
    }
    return status;
}

// ---------------------------------------------------------------- graph form

// Decides after each FP64 residual whether the defect-correction loop goes on,
// with the host loop's rules; sets the WHILE node's condition.
__global__ void k_mixed_check(const LevelScal *__restrict__ ls0, BoxCtl *ctl,
                              cudaGraphConditionalHandle hnd)
{
    ls0 = &MG5_AT(ls0, 0);
    ctl = &MG5_AT(ctl, 0);
    const double rel = ls0->rel;
    const int k = ctl->outer;
    if (k < 64) {
        ctl->hist[k] = rel;
        ctl->nhist = k + 1;
    }
    ctl->rel = rel;
    int stop = 0, status = MG5_E_NOT_CONVERGED;
    if (!isfinite(rel)) {
        stop = 1;
        status = MG5_E_NONFINITE;
    } else if (rel <= ctl->tol) {
        stop = 1;
        status = MG5_OK;
    } else {
        if (rel < ctl->best)
            ctl->best = rel;
        if (k >= 3 && rel > 10.0 * ctl->best) {
            stop = 1;
            status = MG5_E_DIVERGED;
        } else if (k >= ctl->max_outer) {
            stop = 1;
            status = MG5_E_NOT_CONVERGED;
        }
    }
    if (stop) {
        ctl->status = status;
        cudaGraphSetConditional(hnd, 0);
    } else {
        ctl->outer = k + 1;
        cudaGraphSetConditional(hnd, 1);
    }
}

__global__ void k_ctl_init(BoxCtl *ctl, double tol, int max_outer)
{
    ctl = &MG5_AT(ctl, 0);
    ctl->tol = tol;
    ctl->max_outer = max_outer;
    ctl->outer = 0;
    ctl->status = MG5_E_NOT_CONVERGED;
    ctl->nhist = 0;
    ctl->best = INFINITY;
    ctl->rel = 0.0;
}

cudaError_t launch_ctl_init(BoxCtl *ctl, double tol, int max_outer, cudaStream_t st)
{
    k_ctl_init<<<1, 1, 0, st>>>(ctl, tol, max_outer);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_loop_check(const LevelScal *ls0, BoxCtl *ctl, cudaGraphConditionalHandle hnd,
                              cudaStream_t st)
{
    k_mixed_check<<<1, 1, 0, st>>>(ls0, ctl, hnd);
    count_launch(1);
    return cudaGetLastError();
}

int capture_mixed(MixedHier *h, const MixedShared &sh, const double *delta, const mg5_params *p,
                  double *phi, double *grad, BoxCtl *ctl, cudaStream_t st, cudaStream_t st_body,
                  CaptureStats *stats, std::string *err)
{
    RunMix R{h, sh, p, st, err, {}, 0};
    for (int l = 0; l < h->nlev; ++l)
        R.hl[l] = p->h * (double)(1 << l);
    const int inner = inner_cycles_for(p);
    const long long L0 = launches_total();
    cudaStreamCaptureStatus cs;
    cudaGraph_t graph = nullptr;
    CKM(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) {
        *err = "capture_mixed: stream is not capturing";
        return MG5_E_ARG;
    }
    cudaGraphConditionalHandle hnd;
    CKM(cudaGraphConditionalHandleCreate(&hnd, graph, 0, cudaGraphCondAssignDefault));
    k_ctl_init<<<1, 1, 0, st>>>(ctl, p->tol, p->max_cycles);
    CKM(cudaGetLastError());
    const long long n3 = (long long)h->N * h->N * h->N;
    CKM(cudaMemsetAsync(phi, 0, n3 * sizeof(double), st));
    if (int rc = phase_setup(h, sh, delta, p, st, err))
        return rc;
    if (int rc = phase_residual(h, sh, p, phi, st, err, true))   // phi was zeroed above
        return rc;
    k_mixed_check<<<1, 1, 0, st>>>(sh.ls, ctl, hnd);
    CKM(cudaGetLastError());
    // the WHILE node, after everything captured so far on st
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    CKM(cudaStreamGetCaptureInfo(st, &cs, nullptr, &graph, &deps, nullptr, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hnd;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CKM(cudaGraphAddNode(&node, graph, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CKM(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    const long long L1 = launches_total();
    // body: one defect-correction step and the next residual + check
    CKM(cudaStreamBeginCaptureToGraph(st_body, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal));
    RunMix B{h, sh, p, st_body, err, {}, 0};
    for (int l = 0; l < h->nlev; ++l)
        B.hl[l] = R.hl[l];
    int rc = phase_work(B, phi, inner, err);
    if (rc == MG5_OK)
        rc = phase_residual(h, sh, p, phi, st_body, err);
    if (rc == MG5_OK) {
        k_mixed_check<<<1, 1, 0, st_body>>>(sh.ls, ctl, hnd);
        if (cudaGetLastError() != cudaSuccess)
            rc = MG5_E_CUDA;
    }
    cudaGraph_t g_out = nullptr;
    cudaError_t e = cudaStreamEndCapture(st_body, &g_out);
    if (rc != MG5_OK)
        return rc;
    CKM(e);
    const long long L2 = launches_total();
    if (int rc2 = phase_finish(h, sh, phi, st, err))
        return rc2;
    if (grad)
        CKM(launch_force(phi, h->N, h->N, h->N, 0, p->h, 1, grad, st));
    stats->launches_fixed = (L1 - L0) + (launches_total() - L2);
    stats->launches_per_iter = L2 - L1;
    stats->cells_per_iter = B.cu;
    stats->inner = inner;
    stats->cells_fixed = 0;
    return MG5_OK;
}

#undef CKM

}  // namespace mg5
