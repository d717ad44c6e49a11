// mg5_tune.cu -- autotuner of the sweep schedule (host runtime, C ABI in mg5.h).
//
// The smoother's schedule changes speed, not values: the two-pass sweep with
// 32 .. 512 threads per block (by default 256, fewer on coarse grids so that their
// warps reach more SMs), the column march of the mixed mode's FP32 sweep
// (k_march.cu), or the fused plane-march with 8 .. 32 planes per
// CTA, all apply the same cell update to the same snapshot (the sweep of
// Sec. 3.1).  Which is fastest depends on the grid side (waves over the 152
// SMs, shared-memory rings vs L2 reuse) and on the precision (the FP64 sweep
// is bound by the FP64 pipe, the mixed mode's FP32 sweep by issue and
// memory).  The tuner times every candidate on a synthetic field of the side
// with CUDA events (median of repeats after warm-up) and records the fastest
// in a process-wide table keyed by (device, precision, side), which solves,
// batch captures and pooled graphs read when they start.  The table saves to
// and loads from JSON lines keyed by the device's name.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "mg5.h"
#include "mg5_kernels.cuh"

namespace mg5 {
namespace {

using Key = std::tuple<int, int, int>;   // device, precision, side
std::mutex g_tune_mu;
std::map<Key, SweepSchedule> g_tuned;
// bumped on every change of the table: a captured solve records the version it was captured
// under and is not replayed once the table has changed (its launches would follow the old
// schedules, and the schedules change the rounding, not the method)
std::atomic<unsigned long long> g_sched_version{1};

SweepSchedule default_schedule(int precision, int n)
{
    SweepSchedule s;
    s.block = block_spread((long long)n * n * (n / 2));   // coarse grids: smaller blocks, more SMs
    if (precision == MG5_MIXED && march_ok(n))
        s.form = 2;
    else if (precision == MG5_MIXED && fused_ok<float>(n))
        s.form = 1;
    return s;
}

// a smooth periodic field of amplitude amp (phase `salt`) plus a small checkerboard
template <typename T>
__global__ void k_tune_fill(T *a, int n, double amp, int salt)
{
    const long long n3 = (long long)n * n * n;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3)
        return;
    const int k = (int)(t % n), j = (int)((t / n) % n), i = (int)(t / ((long long)n * n));
    const double w = 6.283185307179586 / n;
    const double v = sin(w * (i + salt)) * cos(w * j) + 0.5 * sin(w * (k + 2 * salt)) +
                     0.01 * (((i + j + k) & 1) ? 1.0 : -1.0);
    MG5_AT(a, t) = (T)(amp * v);
}

struct TuneBufs {
    void *in = nullptr, *out = nullptr, *f = nullptr, *B = nullptr;
    double *c = nullptr;
    unsigned long long *clamp = nullptr;
    ~TuneBufs()
    {
        for (void *p : {in, out, f, B, (void *)c, (void *)clamp})
            if (p)
                cudaFree(p);
    }
};

std::vector<SweepSchedule> candidates(int precision, int n)
{
    std::vector<SweepSchedule> v;
    for (int b : {32, 64, 128, 256, 512}) {
        SweepSchedule s;
        s.form = 0;
        s.block = b;
        v.push_back(s);
    }
    const bool fused = precision == MG5_MIXED ? fused_ok<float>(n) : fused_ok<double>(n);
    if (fused)
        for (int c : {8, 16, 32})
            if (c <= n) {
                SweepSchedule s;
                s.form = 1;
                s.chunk = c;
                v.push_back(s);
            }
    if (precision == MG5_MIXED && march_ok(n))
        for (int c : {0, 16, 32, 64, 128})
            if (c <= n) {
                SweepSchedule s;
                s.form = 2;
                s.chunk = c;
                v.push_back(s);
            }
    return v;
}

template <typename T>
cudaError_t time_candidates(int n, int precision, cudaStream_t st, std::vector<SweepSchedule> &cand)
{
    const size_t n3 = (size_t)n * n * n;
    TuneBufs b;
    cudaError_t e = cudaMalloc(&b.in, n3 * sizeof(T));
    if (e == cudaSuccess)
        e = cudaMalloc(&b.out, n3 * sizeof(T));
    if (e == cudaSuccess)
        e = cudaMalloc(&b.f, n3 * sizeof(T));
    const bool base = precision == MG5_MIXED;
    if (e == cudaSuccess && base)
        e = cudaMalloc(&b.B, n3 * sizeof(T));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b.c, sizeof(double));
    if (e == cudaSuccess)
        e = cudaMalloc((void **)&b.clamp, sizeof(unsigned long long));
    if (e != cudaSuccess)
        return e;
    const int g = (int)((n3 + 255) / 256);
    // physical magnitudes of the reduced equation (h = 1, eps ~ 0.01): phi ~ 1, f ~ 1e-2
    k_tune_fill<T><<<g, 256, 0, st>>>((T *)b.in, n, base ? 1e-3 : 1.0, 1);
    k_tune_fill<T><<<g, 256, 0, st>>>((T *)b.f, n, 1e-2, 2);
    if (base)
        k_tune_fill<T><<<g, 256, 0, st>>>((T *)b.B, n, 1.0, 3);
    cudaMemsetAsync(b.c, 0, sizeof(double), st);
    cudaMemsetAsync(b.clamp, 0, sizeof(unsigned long long), st);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const CoefT<T> cf = make_coef<T>(1.0, 0.02);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int warm = 2, reps = 5;
    for (SweepSchedule &s : cand) {
        std::vector<float> ms;
        for (int r = 0; r < warm + reps && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, st);
            e = launch_sweep_sched<T>(s, (const T *)b.in, (T *)b.out, (const T *)b.f, b.c, n, cf,
                                      b.clamp, st, (const T *)b.B);
            cudaEventRecord(e1, st);
            if (e == cudaSuccess)
                e = cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (r >= warm)
                ms.push_back(t);
        }
        if (e != cudaSuccess)
            break;
        std::sort(ms.begin(), ms.end());
        s.ms = ms[ms.size() / 2];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace

unsigned long long schedule_version() { return g_sched_version.load(); }

SweepSchedule sweep_schedule(int device, int precision, int n)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(Key{device, precision, n});
    return it != g_tuned.end() ? it->second : default_schedule(precision, n);
}

bool sweep_tuned(int device, int precision, int n)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tuned.count(Key{device, precision, n}) > 0;
}

// Time every candidate for (current device, precision, n) and record the fastest.
cudaError_t tune_side(int device, int precision, int n, cudaStream_t st, SweepSchedule *out)
{
    std::vector<SweepSchedule> cand = candidates(precision, n);
    cudaError_t e = precision == MG5_MIXED ? time_candidates<float>(n, precision, st, cand)
                                           : time_candidates<double>(n, precision, st, cand);
    if (e != cudaSuccess)
        return e;
    const SweepSchedule best =
        *std::min_element(cand.begin(), cand.end(),
                          [](const SweepSchedule &a, const SweepSchedule &b) { return a.ms < b.ms; });
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[Key{device, precision, n}] = best;
        ++g_sched_version;
    }
    if (out)
        *out = best;
    return cudaSuccess;
}

}  // namespace mg5

using namespace mg5;

namespace {

std::string device_name(int device)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string s = prop.name;
    for (char &c : s)
        if (c == '"' || c == '\\')
            c = '_';
    return s;
}

}  // namespace

extern "C" {

int mg5_schedule_get(int device, int precision, int n, mg5_schedule *out)
{
    if (!out || (precision != MG5_FP64 && precision != MG5_MIXED) || n < 1)
        return MG5_E_ARG;
    const SweepSchedule s = sweep_schedule(device, precision, n);
    out->form = s.form;
    out->block = s.block;
    out->chunk = s.chunk;
    out->ms = s.ms;
    return sweep_tuned(device, precision, n) ? MG5_OK : MG5_W_UNTUNED;
}

int mg5_schedule_set(int device, int precision, int n, const mg5_schedule *s)
{
    if (!s || (precision != MG5_FP64 && precision != MG5_MIXED) || n < 1)
        return MG5_E_ARG;
    if ((s->form != MG5_SWEEP_TWO_PASS && s->form != MG5_SWEEP_FUSED &&
         s->form != MG5_SWEEP_MARCH) || s->block < 32 ||
        s->block > 1024 || s->block % 32 || s->chunk < 0)
        return MG5_E_ARG;
    SweepSchedule v;
    v.form = s->form;
    v.block = s->block;
    v.chunk = s->chunk;
    v.ms = s->ms;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[Key{device, precision, n}] = v;
    ++g_sched_version;
    return MG5_OK;
}

int mg5_tune_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    ++g_sched_version;
    return MG5_OK;
}

int mg5_tune_save(const char *path)
{
    if (!path)
        return MG5_E_ARG;
    std::vector<std::pair<Key, SweepSchedule>> rows;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        rows.assign(g_tuned.begin(), g_tuned.end());
    }
    FILE *fp = std::fopen(path, "w");
    if (!fp)
        return MG5_E_ARG;
    for (const auto &r : rows) {
        const SweepSchedule &s = r.second;
        std::fprintf(fp,
                     "{\"gpu\": \"%s\", \"precision\": \"%s\", \"n\": %d, \"form\": \"%s\", "
                     "\"block\": %d, \"chunk\": %d, \"ms\": %.6g}\n",
                     device_name(std::get<0>(r.first)).c_str(),
                     std::get<1>(r.first) == MG5_MIXED ? "mixed" : "fp64", std::get<2>(r.first),
                     s.form == 2 ? "march" : (s.form == 1 ? "fused" : "two-pass"), s.block,
                     s.chunk, (double)s.ms);
    }
    return std::fclose(fp) == 0 ? MG5_OK : MG5_E_ARG;
}

// Reads the lines mg5_tune_save writes; entries for GPUs of another name are skipped.
// Returns the number of entries applied, or MG5_E_ARG for an unreadable file or line.
int mg5_tune_load(const char *path)
{
    if (!path)
        return MG5_E_ARG;
    FILE *fp = std::fopen(path, "r");
    if (!fp)
        return MG5_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        ndev = 0;
    }
    std::vector<std::string> names;
    for (int d = 0; d < ndev; ++d)
        names.push_back(device_name(d));
    char line[512];
    int applied = 0, bad = 0;
    while (std::fgets(line, sizeof line, fp)) {
        if (line[0] == '\n' || line[0] == 0)
            continue;
        char gpu[256] = {}, prec[16] = {}, form[16] = {};
        int n = 0, block = 0, chunk = 0;
        double ms = 0.0;
        if (std::sscanf(line,
                        "{\"gpu\": \"%255[^\"]\", \"precision\": \"%15[^\"]\", \"n\": %d, "
                        "\"form\": \"%15[^\"]\", \"block\": %d, \"chunk\": %d, \"ms\": %lf}",
                        gpu, prec, &n, form, &block, &chunk, &ms) != 7) {
            ++bad;
            continue;
        }
        mg5_schedule s;
        s.form = std::strcmp(form, "march") == 0
                     ? MG5_SWEEP_MARCH
                     : (std::strcmp(form, "fused") == 0 ? MG5_SWEEP_FUSED : MG5_SWEEP_TWO_PASS);
        s.block = block;
        s.chunk = chunk;
        s.ms = (float)ms;
        const int p = std::strcmp(prec, "mixed") == 0 ? MG5_MIXED : MG5_FP64;
        for (int d = 0; d < ndev; ++d)
            if (names[d] == gpu && mg5_schedule_set(d, p, n, &s) == MG5_OK)
                ++applied;
    }
    std::fclose(fp);
    return bad ? MG5_E_ARG : applied;
}

}  // extern "C"
