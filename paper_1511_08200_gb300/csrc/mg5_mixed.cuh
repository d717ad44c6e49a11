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
    float2 *spec[2] = {};               // coarsest-grid DFT work (coarsest side >= kSpectralMinSide)
    size_t bytes = 0;
};

// Context resources the mixed solve borrows.
struct MixedShared {
    double2 *partials;
    LevelScal *ls;   // slot 0: FP64 finest; slots kInnerBase + l: inner grids
    SolveCounters *cnt;
    double *h_rel;   // pinned host scalar
    Profiler *prof;
    cudaEvent_t wait_ev = nullptr;   // blocking-sync event for host waits (nullptr: spin on the stream)
};

// FP32 V-cycles per FP64 defect-correction step: the caller's count, else 4 below
// a relative tolerance of 1e-7 and 3 above.  Measured at 512^3: a step of 3 cycles
// reduces the residual ~2e-3, of 4 ~6e-5 (FP32 bounds a step near 3e-5), so 1e-8
// takes two steps of 4 (8 cycles, 3 FP64 residuals) instead of three of 3 (9, 4).
inline int inner_cycles_for(const mg5_params *p)
{
    if (p->inner_cycles > 0)
        return p->inner_cycles;
    return p->tol < 1e-7 ? 4 : 3;
}

// Wait until st has drained: sleep on `ev` (a blocking-sync event) when given, else spin.
inline cudaError_t host_wait(cudaStream_t st, cudaEvent_t ev)
{
    if (!ev)
        return cudaStreamSynchronize(st);
    cudaError_t e = cudaEventRecord(ev, st);
    return e == cudaSuccess ? cudaEventSynchronize(ev) : e;
}

// Per-box loop control of the graph form (device memory).
struct BoxCtl {
    double tol;
    int max_outer;
    int outer;       // defect-correction steps done
    int status;
    int nhist;
    double best;
    double rel;
    double hist[64];
};

// What one captured solve costs per WHILE iteration (host bookkeeping).
struct CaptureStats {
    long long launches_fixed;     // kernels outside the loop
    long long launches_per_iter;  // kernels of one loop body
    long long cells_per_iter;     // cell updates of one loop body (coarsest grids excluded)
    int inner;
    long long cells_fixed;        // cell updates outside the loop (FP64 form: start and first smoothing)
};

// The graph form's loop control (mg5_mixed.cu): reset the control block; after each
// finest-grid residual record it and set the WHILE condition by the host loop's rules
// (stop at rel <= tol, on a non-finite or diverging residual, or after max_outer checks).
cudaError_t launch_ctl_init(BoxCtl *ctl, double tol, int max_outer, cudaStream_t st);
cudaError_t launch_loop_check(const LevelScal *ls0, BoxCtl *ctl, cudaGraphConditionalHandle hnd,
                              cudaStream_t st);

size_t mixed_bytes(int N);
int alloc_mixed(int N, size_t budget, size_t *held, MixedHier **out, std::string *err);
void free_mixed(MixedHier *m, size_t *held);
// phi: device FP64 N^3 initial guess in, mean-zero solution out.
// zero_start: phi holds zeros (not a warm start), so the first residual skips the stencil
int solve_mixed(MixedHier *m, const MixedShared &sh, const double *delta, const mg5_params *p,
                double *phi, mg5_info *info, cudaStream_t st, std::string *err, bool zero_start);
// Record, into the graph being captured on `st`, a whole mixed solve (phi
// zero start) with its defect-correction loop as a WHILE node whose body is
// captured on `st_body`; then gauge and (if grad) the force.  The loop state
// lands in *ctl.
int capture_mixed(MixedHier *m, const MixedShared &sh, const double *delta, const mg5_params *p,
                  double *phi, double *grad, BoxCtl *ctl, cudaStream_t st, cudaStream_t st_body,
                  CaptureStats *stats, std::string *err);

}  // namespace mg5
