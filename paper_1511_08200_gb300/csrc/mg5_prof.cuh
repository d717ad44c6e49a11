// mg5_prof.cuh -- optional per-kernel-class timing with CUDA events recorded
// on the launching stream (internal).  Off by default; when on, every timed
// launch site records an event pair and the pairs are resolved after the
// entry point has synchronised its stream.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace mg5 {

enum ProfKernel {
    PK_SWEEP64 = 0,      // one full snapshot red-black sweep on the finest grid, FP64 (2 launches)
    PK_RESTRICT64,       // residual + 8-child restriction, FP64
    PK_COARSE_RHS64,
    PK_PROLONG64,
    PK_COARSEST64,
    PK_SWEEP32,          // correction-form sweep, FP32 (2 launches)
    PK_RESTRICT32,
    PK_COARSE_RHS32,
    PK_PROLONG32,
    PK_COARSEST32,
    PK_RESID64_MIXED,    // FP64 residual of the defect-correction loop
    PK_UPDATE_MIXED,
    PK_PATCH_SWEEP,      // Dirichlet patch sweep, FP64 (2 launches)
    PK_PATCH_RESID,
    PK_FORCE,
    PK_REFINE,
    PK_REDUCE,           // finalize / sums / scale / gauge
    PK_SWEEP64C,         // the same sweeps on the coarse grids of the hierarchy
    PK_SWEEP32C,
    PK_PATCH_SWEEPC,
    PK_COUNT
};

struct Profiler {
    bool on = false;
    struct Pending {
        int kid;
        cudaEvent_t a, b;
        double units;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[PK_COUNT] = {};
    long long calls[PK_COUNT] = {};
    double units[PK_COUNT] = {};   // cells processed (class-specific unit)

    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    // record the start of a timed launch; returns the slot index or -1
    int begin(int kid, cudaStream_t st, double u)
    {
        if (!on)
            return -1;
        Pending p{kid, get(), get(), u};
        cudaEventRecord(p.a, st);
        pending.push_back(p);
        return (int)pending.size() - 1;
    }
    void end(int slot, cudaStream_t st)
    {
        if (slot >= 0)
            cudaEventRecord(pending[slot].b, st);
    }
    // after the stream has synchronised
    void resolve()
    {
        for (Pending &p : pending) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
                ms[p.kid] += t;
                calls[p.kid] += 1;
                units[p.kid] += p.units;
            }
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
        cudaGetLastError();
    }
    void reset()
    {
        for (int k = 0; k < PK_COUNT; ++k) {
            ms[k] = 0.0;
            calls[k] = 0;
            units[k] = 0.0;
        }
    }
    void destroy()
    {
        for (Pending &p : pending) {
            pool.push_back(p.a);
            pool.push_back(p.b);
        }
        pending.clear();
        for (cudaEvent_t e : pool)
            cudaEventDestroy(e);
        pool.clear();
    }
};

// RAII scope: times the launches issued while it lives.
struct ProfScope {
    Profiler *p;
    int slot;
    cudaStream_t st;
    ProfScope(Profiler *p_, int kid, cudaStream_t st_, double units = 0.0)
        : p(p_), slot(p_ ? p_->begin(kid, st_, units) : -1), st(st_)
    {
    }
    ~ProfScope()
    {
        if (p)
            p->end(slot, st);
    }
};

}  // namespace mg5
