// mg5_mixed.cuh -- mixed-precision solve (internal): an FP64 residual and
// defect-correction outer loop around FP32 FAS V-cycles that solve the
// correction equation  op(B + e) - op(B) = r  with B = fp32(phi).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "mg5.h"
#include "mg5_kernels.cuh"
#include "mg5_prof.cuh"

namespace mg5 {

constexpr int kMixMaxLevels = 16;

struct MixedHier {
    int N = 0;
    int nlev = 0;
    int n[kMixMaxLevels] = {};
    double *f64 = nullptr;              // s delta, FP64, finest grid
    float *B[kMixMaxLevels] = {};       // base fp32(phi) and its restrictions
    float *e[kMixMaxLevels] = {};       // correction iterate
    float *etmp[kMixMaxLevels] = {};    // ping-pong partner
    float *f[kMixMaxLevels] = {};       // right-hand side of the correction equation
    float *e0[kMixMaxLevels] = {};      // restricted correction before the coarse solve
    size_t bytes = 0;
};

// Context resources the mixed solve borrows.
struct MixedShared {
    double2 *partials;
    LevelScal *ls;   // slot 0: FP64 finest; slots kInnerBase + l: inner grids
    SolveCounters *cnt;
    double *h_rel;   // pinned host scalar
    Profiler *prof;
};

size_t mixed_bytes(int N);
int alloc_mixed(int N, size_t budget, size_t *held, MixedHier **out, std::string *err);
void free_mixed(MixedHier *m, size_t *held);
// phi: device FP64 N^3 initial guess in, mean-zero solution out.
int solve_mixed(MixedHier *m, const MixedShared &sh, const double *delta, const mg5_params *p,
                double *phi, mg5_info *info, cudaStream_t st, std::string *err);

}  // namespace mg5
