// mg5_kernels.cuh -- host-side launchers of the mg5 kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "mg5.h"
#include "mg5_dev.cuh"

namespace mg5 {

// Device scalars of one grid of the hierarchy.
struct LevelScal {
    double c;      // compatibility constant
    double m;      // mean of the last residual (before projection)
    double rnorm;  // ||r - m||_2 of the last residual
    double rel;    // rnorm / fnorm (finest grid) or rnorm
    double fnorm;  // ||f||_2 (finest grid)
    double mean;   // scratch for the gauge (mean of phi)
    double pad[2];
};

// Device counters shared by one solve.
struct SolveCounters {
    unsigned long long clamped;
    int coarse_sweeps;
    int pad;
};

constexpr int kBlock = 256;
constexpr int kScalSlots = 48;   // LevelScal slots held by a context
constexpr int kPatchSlot = 16;   // slot used by the patch relaxation
constexpr int kStepSlot = 17;    // slot used by the single-step entry points
constexpr int kInnerBase = 20;   // first slot of the mixed solve's FP32 grids
constexpr int kMaxPartials = 8192;  // partial-sum slots (double2) per reduction; the last one
                                    // holds the last-block counter of the in-kernel finalize
// blocks of a residual-statistics reduction: each writes one Moments (two slots), and the
// Moments that would share the counter's slot is left out
constexpr int kMomentBlocks = kMaxPartials / 2 - 1;
// Grid caps of the reduction kernels (grid-stride loops).  The one-block finalize spends
// FP64 instructions on every partial, and FP64 runs at 1/64 of the FP32 rate here, so
// the partials are kept few: FP64-bound producers use 4 blocks of 256 per SM (152 SMs),
// the others 8 (one full wave).
constexpr int kReduceBlocksFp64 = 4 * 152;
constexpr int kReduceBlocks = 8 * 152;
static_assert(kReduceBlocks <= kMomentBlocks, "partials buffer too small");

// Number of blocks of kBlock threads to cover `work` items (capped for reductions).
inline int blocks_for(long long work) { return (int)((work + kBlock - 1) / kBlock); }

constexpr int kSMs = 152;   // GB300: 2 dies x 76 SMs

// Threads per block for a grid of `work` threads: kBlock while that still gives every SM two
// blocks, else fewer (a multiple of 32, at least one warp), so that a coarse grid's warps reach
// more SMs.  GB300 runs FP64 at 2 lanes a clock per SM: an FP64 kernel on a small grid takes as
// long as the warps its busiest SM holds need, not as long as its work needs over the GPU.
inline int block_spread(long long work)
{
    const long long per = work / (2 * kSMs);
    if (per >= kBlock)
        return kBlock;
    const int b = (int)(per & ~31ll);
    return b < 32 ? 32 : b;
}
// The FP64 residual + restriction kernels (domain and patch) run a thread per fine cell on
// grids of up to this many fine cells, a thread per coarse cell above.
constexpr long long kChildMaxFine = 32 * 32 * 32;

// Blocks of block_spread(work) threads that cover `work` threads.
inline int grid_spread(long long work)
{
    const int b = block_spread(work);
    return (int)((work + b - 1) / b);
}

// The smoother's relaxation weight of a parameter set (0 selects the default: 1.3 for the FP64
// solves, whose V-cycle count it cuts; 1 for the mixed mode, whose inner cycle count is fixed
// and whose FP32 correction sweeps gain nothing from it).
inline double omega_of(const mg5_params *p)
{
    if (p->omega > 0.0)
        return p->omega;
    return p->precision == MG5_FP64 ? 1.3 : 1.0;
}

// Process-wide count of kernel launches the library has enqueued.
void count_launch(long long n);
long long launches_total();

// finalize modes
// FIN_RESID: m = mean r, c -= m, rnorm = ||r - m||, rel = rnorm / fnorm; the partials
//            are Moments (count, mean, M2) per block, combined pairwise
// FIN_STATS: as FIN_RESID but c is left alone
// FIN_NORM:  rnorm = ||r|| (no projection), rel = rnorm / fnorm
// FIN_FNORM: fnorm = sqrt(sum of the second component)
// FIN_MEAN:  mean = sum of the first component / ncells
enum FinalizeMode { FIN_RESID = 0, FIN_FNORM = 1, FIN_MEAN = 2, FIN_STATS = 3, FIN_NORM = 4 };

// A reduction finalized by the last block of its own kernel (mg5_fin.cuh) instead of a
// separate launch_finalize: the grid size is the number of partials.  ls == nullptr: no
// finalize in the kernel.  The partial buffer's last slot holds the blocks-done counter
// (zero between launches; buffers are zeroed when allocated).
struct Fin {
    LevelScal *ls = nullptr;
    int mode = 0;
    double ncells = 0.0;
};

// ---- FP64/FP32 periodic kernels (templates instantiated for double and float)
// B (optional): base field of the correction form (mixed precision)
// two-pass sweep (red kernel, black kernel) with `block` threads per block
template <typename T>
cudaError_t launch_sweep(const T *in, T *out, const T *f, const double *cptr, int n,
                         CoefT<T> cf, unsigned long long *clamp, cudaStream_t st,
                         const T *B = nullptr, int block = kBlock);
// fused red+black sweep (k_fused.cu): one read and one write of phi per cell; each CTA
// marches over `chunk` planes (0: enough CTAs for several waves)
template <typename T>
cudaError_t launch_sweep_fused(const T *in, T *out, const T *f, const double *cptr, int n,
                               CoefT<T> cf, unsigned long long *clamp, cudaStream_t st,
                               const T *B = nullptr, int chunk = 0);
constexpr int kFusedMinN = 32;   // smaller grids use the two-pass sweep
// the fused kernel needs 16-byte row chunks: n a multiple of 16 / sizeof(T)
template <typename T>
inline bool fused_ok(int n)
{
    return n >= kFusedMinN && n % (int)(16 / sizeof(T)) == 0;
}
cudaError_t prepare_fused_kernels();
// FP32 correction-form sweep as a column march (k_march.cu): 16 x 32 tiles, n a multiple
// of 32, B required; `chunk` planes per CTA (0: about six waves of two CTAs per SM)
bool march_ok(int n);
cudaError_t launch_sweep_march(const float *in, float *out, const float *f, const float *B,
                               const double *cptr, int n, CoefT<float> cf,
                               unsigned long long *clamp, cudaStream_t st, int chunk = 0);
cudaError_t prepare_march_kernel();

// How one grid side is swept (speed only: every schedule computes the same values).
struct SweepSchedule {
    int form = 0;     // 0: two-pass, 1: fused, 2: column march (FP32 correction form)
    int block = kBlock;
    int chunk = 0;
    float ms = 0.f;   // tuned time of one sweep (0: not measured)
};
// The schedule of (device, precision, side): the tuned one, else the default
// (FP64 two-pass; the mixed mode's FP32 correction form as a column march on sides that are
// multiples of 32, else fused where it fits).
SweepSchedule sweep_schedule(int device, int precision, int n);
// Changes with every change of the schedule table (captured solves record it; mg5_tune.cu).
unsigned long long schedule_version();
bool sweep_tuned(int device, int precision, int n);
// time the candidates for (device, precision, n) on st and record the fastest (mg5_tune.cu)
cudaError_t tune_side(int device, int precision, int n, cudaStream_t st, SweepSchedule *out);
template <typename T>
cudaError_t launch_sweep_sched(const SweepSchedule &s, const T *in, T *out, const T *f,
                               const double *cptr, int n, CoefT<T> cf, unsigned long long *clamp,
                               cudaStream_t st, const T *B = nullptr)
{
    if constexpr (sizeof(T) == 4) {
        if (s.form == 2 && B && march_ok(n))
            return launch_sweep_march(in, out, f, B, cptr, n, cf, clamp, st, s.chunk);
    }
    if ((s.form == 1 || s.form == 2) && fused_ok<T>(n))
        return launch_sweep_fused<T>(in, out, f, cptr, n, cf, clamp, st, B, s.form == 1 ? s.chunk : 0);
    return launch_sweep<T>(in, out, f, cptr, n, cf, clamp, st, B, s.block);
}
template <typename T>
cudaError_t launch_operator(const T *phi, int n, CoefT<T> cf, T *out, cudaStream_t st);
// r (nullable) = f + c - op(phi); partial sums (sum r, sum r^2) per block.
template <typename T>
cudaError_t launch_residual(const T *phi, const T *f, const double *cptr, int n, CoefT<T> cf,
                            T *r, double2 *partials, int *nblocks, cudaStream_t st,
                            const Fin &fin = Fin());
// fused residual + 8-child restriction of v and r (vc and v0c get R v, rc gets R r).
template <typename T>
cudaError_t launch_resid_restrict(const T *v, const T *f, const double *cptr, int n,
                                  CoefT<T> cf, T *vc, T *v0c, T *rc, double2 *partials,
                                  int *nblocks, cudaStream_t st, const T *B = nullptr,
                                  const Fin &fin = Fin());
// the same for the FP32 correction form (B required) as a column march (k_march_resid.cu):
// n a multiple of 32; the coarse values equal the gather kernel's to the bit
// The bottom of a V-cycle in one CTA (k_bottom.cu): the visit of grid a (side na <= 8) and
// the solve of the coarsest grid b = na / 2 below it, for periodic grids; Ba/Bb the bases of
// the mixed mode's correction form (both or neither).
bool bottom_ok(int na);
template <typename T>
cudaError_t launch_bottom(T *va, const T *fa, const T *Ba, const T *Bb, int na, CoefT<T> cfa,
                          CoefT<T> cfb, const LevelScal *ls_up, LevelScal *lsa, LevelScal *lsb,
                          int nu1, int nu2, int nu_coarse, double rtol, unsigned long long *clamp,
                          int *sweeps, cudaStream_t st);
bool resid_march_ok(int n);
cudaError_t prepare_resid_march_kernel();
cudaError_t launch_resid_restrict_march(const float *e, const float *f, const double *cptr, int n,
                                        CoefT<float> cf, float *vc, float *v0c, float *rc,
                                        double2 *partials, int *nblocks, cudaStream_t st,
                                        const float *B, const Fin &fin = Fin());
// coarse = 8-child mean of fine
template <typename T>
cudaError_t launch_restrict(const T *fine, int n, T *coarse, cudaStream_t st);
// fc = op_c(vc) + fc - m_fine ; c_coarse = 0
template <typename T>
cudaError_t launch_coarse_rhs(const T *vc, T *fc, const double *m_fine, double *c_coarse, int nc,
                              CoefT<T> cfc, cudaStream_t st, const T *B = nullptr);
// vf += P(vc - v0c) (v0c may be NULL: plain prolongation of vc); c_fine += c_coarse if both non-NULL
template <typename T>
cudaError_t launch_prolong_add(const T *vc, const T *v0c, int nc, T *vf, double *c_fine,
                               const double *c_coarse, cudaStream_t st);
// coarsest grids of more than kSpectralMinSide^3 cells (k_spectral.cu): `iters` times the
// residual, its exact periodic-Laplacian solve by DFT added, two red-black sweeps; w0, w1 are
// complex work arrays of n^3 (double2 for T = double, float2 for float)
constexpr int kSpectralMinSide = 7;
constexpr int kSpectralIters = 4;
template <typename T>
cudaError_t launch_coarsest_spectral(T *v, T *tmp, const T *f, int n, CoefT<T> cf, LevelScal *ls,
                                     int iters, unsigned long long *clamp, int *sweeps,
                                     double2 *partials, void *w0, void *w1, cudaStream_t st,
                                     const T *B = nullptr);
// coarsest grid: sweeps until the residual falls by rtol or nu_max sweeps; one CTA.
template <typename T>
cudaError_t launch_coarsest(T *v, T *tmp, const T *f, int n, CoefT<T> cf, double *cptr, int nu_max,
                            double rtol, unsigned long long *clamp, int *sweeps, cudaStream_t st,
                            const T *B = nullptr);

// ---- FP64 helpers
cudaError_t launch_finalize(const double2 *partials, int nb, double ncells, LevelScal *ls,
                            int mode, cudaStream_t st);
// f = s * delta + add (add read from add_dev on the device when given), partial sums (0, (s delta)^2)
cudaError_t launch_scale(const double *delta, double s, double *f, long long n3, double2 *partials,
                         int *nblocks, cudaStream_t st, double add = 0.0,
                         const double *add_dev = nullptr, const Fin &fin = Fin());
// partial sums (phi, 0)
cudaError_t launch_sum(const double *phi, long long n3, double2 *partials, int *nblocks,
                       cudaStream_t st, const Fin &fin = Fin());
// phi -= *mean
cudaError_t launch_sub_mean(double *phi, long long n3, const double *mean, cudaStream_t st);
cudaError_t launch_force(const double *phi, int d0, int d1, int d2, int ghost, double h,
                         int periodic, double *grad, cudaStream_t st);
cudaError_t launch_refine(const double *phic, int nc, const int o[3], const int pn[3], int ghost,
                          double *fine, cudaStream_t st);
// tricubic variant (4-point Lagrange per axis), periodic source
cudaError_t launch_refine_cubic(const double *phic, int nc, const int o[3], const int pn[3],
                                int ghost, double *fine, cudaStream_t st);
// the same interpolation from a box of dims bd whose interior starts at offset pg (no wrap)
cudaError_t launch_refine_box(const double *box, const int bd[3], int pg, const int o[3],
                              const int pn[3], int ghost, double *fine, cudaStream_t st);
// Dirichlet patch (interior pf, box pf + 2): one full sweep in -> out (out must hold the ghosts).
// With v0 (coarse patch grids) the ghosts of out follow each half-sweep by the extrapolated
// boundary condition of weight w (k_patch.cu), written by the threads of their anchor cells.  mask (interior-indexed, optional):
// cells with mask 0 are not relaxed and keep their values.
cudaError_t launch_patch_sweep(const double *in, double *out, const double *fint, double rhs_add,
                               const int pf[3], CoefT<double> cf, unsigned long long *clamp,
                               cudaStream_t st, const double *v0 = nullptr, double w = 0.0,
                               const unsigned char *mask = nullptr);
// partial sums (r, r^2) of r = fint + rhs_add - op(phi) over the interior (the cells of mask)
cudaError_t launch_patch_residual(const double *phi, const double *fint, double rhs_add,
                                  const int pf[3], CoefT<double> cf, double2 *partials, int *nblocks,
                                  cudaStream_t st, const unsigned char *mask = nullptr,
                                  const Fin &fin = Fin());

// ---- Dirichlet patch multigrid (k_patch.cu); p = fine interior dims, q = coarse interior dims
// mask (fine, optional): the residual of cells with mask 0 counts as zero
cudaError_t launch_pbox_resid_restrict(const double *v, const double *f, const int p[3],
                                       CoefT<double> cf, double *vc, double *v0c, double *fc,
                                       double2 *partials, int *nblocks, cudaStream_t st,
                                       const unsigned char *mask = nullptr,
                                       const Fin &fin = Fin());
cudaError_t launch_pbox_coarse_rhs(const double *vc, double *fc, const int q[3], CoefT<double> cf,
                                   cudaStream_t st);
// mask (fine, optional): only cells with mask != 0 take the correction
cudaError_t launch_pbox_prolong(const double *vc, const double *v0c, const int q[3], double *vf,
                                cudaStream_t st, const unsigned char *mask = nullptr);
cudaError_t launch_pbox_ghosts(const double *fine_box, const int p[3], double *g1, double *g2,
                               double *g3, cudaStream_t st);
cudaError_t launch_pbox_coarsest(double *A, double *B, const double *f, const int p[3],
                                 CoefT<double> cf, int nu_max, double rtol, unsigned long long *clamp,
                                 int *sweeps, cudaStream_t st, const double *v0 = nullptr,
                                 double w = 0.0, const unsigned char *mask = nullptr);

// ---- position-dependent truncation (k_mask.cu)
// coarse mask (interior q = p/2) = 1 where all 8 children have mask != 0
cudaError_t launch_mask_restrict(const unsigned char *mf, const int p[3], unsigned char *mc,
                                 cudaStream_t st);
// f = s delta + add on every cell; partial sums (number of cells of mask, (s delta)^2 over them)
cudaError_t launch_scale_masked(const double *delta, double s, double *f, long long n,
                                const unsigned char *mask, double2 *partials, int *nblocks,
                                cudaStream_t st, double add);
// mask of the (2 pn) fine interior: |grad phi / 2| > theta |grad Psi_GR| at the parent cell
// (parent grid of dims pd, periodic or a refinement's interior)
cudaError_t launch_parent_force_mask(const double *grad_phi, const double *grad_gr, const int pd[3],
                                     int periodic, const int o[3], const int pn[3], double theta,
                                     unsigned char *mask, unsigned long long *count,
                                     cudaStream_t st);

}  // namespace mg5
