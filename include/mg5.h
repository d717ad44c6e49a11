/*
 * mg5.h -- C ABI of the GB300 (sm_103a) nonlinear multigrid library for the
 * nDGP fifth force.
 *
 * Paper: Barreira, Bose & Li, "Speeding up N-body simulations of modified
 * gravity: Vainshtein screening models", arXiv:1511.08200.
 *
 * The library solves Eq. (eomvarphi),
 *     lap(phi) + alpha [ (lap phi)^2 - (d_i d_j phi)^2 ] = s delta,
 * alpha = r_c^2 / (3 beta a^2), s = 8 pi G a^2 rho_bar / (3 beta), on a
 * periodic, uniform, cell-centred grid (the domain level of Sec. 3.1), by
 * FAS multigrid V-cycles whose smoother solves each cell's equation exactly
 * (the fixed point of the Newton update, Eq. newton).  It also provides the
 * speed-up of Sec. 3.2: fine-level phi interpolated from the coarse level
 * (mg5_refine_interpolate) instead of relaxed (mg5_relax_patch), and the
 * force by central differences of phi at cell centres (mg5_force).
 *
 * Conventions shared by every entry point
 *   - Fields are C-order arrays, index (i*N1 + j)*N2 + k, k fastest, i <-> x.
 *   - Pointers to fields are DEVICE pointers (cudaMalloc / torch CUDA
 *     tensors) unless MG5_HOST_IO is set where documented.  The caller owns
 *     every input and output buffer; the context owns its scratch memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     enqueued on it; entry points that need a scalar on the host (the
 *     convergence test) synchronise that stream and say so.
 *   - Every entry point returns an mg5 status code; nothing is thrown across
 *     the ABI.  On MG5_E_CUDA the text of the CUDA error is available from
 *     mg5_last_error().
 *   - Discrete operator (the reading of the paper's unstated discretisation):
 *     D_aa = (phi[+e_a] + phi[-e_a] - 2 phi) / h^2,
 *     D_ab = (phi[+a+b] - phi[+a-b] - phi[-a+b] + phi[-a-b]) / (4 h^2),
 *     L = sum D_aa, (d_i d_j phi)^2 = sum D_aa^2 + 2 sum_{a<b} D_ab^2.
 *   - On a periodic grid the discrete nonlinear term has a non-zero mean, so
 *     the library solves  op(phi) = s delta + c  with mean(phi) = 0 and a
 *     scalar c (the compatibility constant, reported in mg5_info).
 * One context per host thread, or external locking.
 */
#ifndef MG5_H
#define MG5_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define MG5_OK               0
#define MG5_W_DISC_CLAMP     1   /* converged, but some cell had no real root (clamped, counted) */
#define MG5_W_UNTUNED        2   /* mg5_schedule_get: no tuned entry, *out is the default */
#define MG5_E_ARG           -1   /* bad size, pointer or parameter */
#define MG5_E_OOM           -2   /* scratch would exceed the context's HBM budget */
#define MG5_E_CUDA          -3   /* a CUDA call failed; see mg5_last_error */
#define MG5_E_NOT_CONVERGED -4   /* max_cycles reached; phi holds the last iterate */
#define MG5_E_DIVERGED      -5   /* residual grew 10x above its best after >= 3 cycles */
#define MG5_E_NONFINITE     -6   /* NaN or Inf in the residual */
#define MG5_E_TOO_LARGE     -7   /* the grid exceeds an entry point's fixed scratch */

/* ------------------------------------------------------------ precision */
#define MG5_FP64  0   /* every kernel in FP64 */
#define MG5_MIXED 1   /* FP64 residual + defect-correction outer loop around FP32 V-cycles */

/* ------------------------------------------------------------ flags */
#define MG5_WARM     1u   /* phi holds the initial guess (Sec. 3.1: zero or the previous step) */
#define MG5_HOST_IO  2u   /* delta, phi, grad are HOST pointers; the library copies them */
#define MG5_FMG      4u   /* MG5_FP64 from zero: full-multigrid start (rhs restricted down, coarsest
                             solved, one V-cycle per finer grid on the interpolated solution) */
#define MG5_GRAPH    8u   /* A solve from zero as ONE CUDA-graph launch: the context captures, per
                             (N, parameters, grad or not, MG5_FMG or not), the whole solve with its
                             loop (MG5_MIXED: the defect correction; MG5_FP64: the V-cycle) as a
                             device-controlled WHILE node, with its own hierarchy and staging
                             buffers, and replays it (copy in, launch, copy out, one sync): the same
                             kernels as the host-driven solve, without a host round trip per cycle.
                             Not with MG5_WARM (with MG5_HOST_IO the host buffers are staged in and
                             out around the replay); MG5_FP64 needs nu1 + nu2 even and
                             N with two grids or more (MG5_E_ARG otherwise).  A change of the
                             sweep-schedule table (mg5_autotune, mg5_schedule_set,
                             mg5_tune_clear, mg5_tune_load) retires the captured solves and
                             batches: the next call captures again under the new schedules. */

typedef struct mg5_ctx mg5_ctx;  /* opaque; owns the device hierarchy, resident between calls */

/* Solver parameters.  alpha, s: coefficients of Eq. (eomvarphi) (see
 * mg5_ndgp_coefficients); h: cell size; tol: stop when
 * ||r - mean r||_2 <= tol ||s delta||_2 on the finest grid (the norm is reduced
 * from sums of deviations from a residual value of the same set, so it stays
 * accurate when |mean r| is far above the spread of r).
 * nu1, nu2: pre-/post-smoothing sweeps; nu_coarse: sweep cap on the
 * coarsest grid (which sweeps until its residual falls 1e-3);
 * max_cycles: V-cycle cap (MG5_MIXED: cap on FP64 defect-correction steps);
 * precision: MG5_FP64 or MG5_MIXED.
 * omega: relaxation weight of every smoothing update, v <- v + omega (v_GS - v) with v_GS the
 * cell's exact root (Eq. newton's fixed point); 1 is the plain nonlinear Gauss-Seidel update.
 * 0 selects the default: 1.3 for MG5_FP64 (a V(2,2) cycle then reduces the residual ~0.02
 * instead of ~0.09; same converged solution), 1 for MG5_MIXED (its inner cycle count is fixed,
 * so the weight buys nothing there).  Valid: 0 <= omega < 2. */
typedef struct {
    double alpha, s, h, tol;
    int nu1, nu2, nu_coarse, max_cycles;
    int precision;
    int inner_cycles;   /* MG5_MIXED: FP32 V-cycles per FP64 step (0 = 4 if tol < 1e-7, else 3) */
    double omega;       /* smoother relaxation weight (0 = default: 1.3 FP64, 1 mixed) */
} mg5_params;

/* Per-solve report, written on return (after the stream has synchronised). */
typedef struct {
    int status;              /* same as the return code */
    int cycles;              /* V-cycles with coarse correction (all inner cycles in MG5_MIXED) */
    int outer_iters;         /* MG5_MIXED: FP64 defect-correction steps; 0 otherwise */
    int levels;              /* grids in the hierarchy */
    int coarsest_n;          /* side of the coarsest grid */
    int n_history;           /* valid entries of history */
    double rel_residual;     /* final ||r - mean r||_2 / ||s delta||_2 (FP64) */
    double compat_c;         /* compatibility constant c of the finest grid */
    double phi_mean_removed; /* mean subtracted from phi at the end */
    long long disc_clamped;  /* cells whose discriminant was clamped */
    long long cell_updates;  /* cells relaxed: one per cell per full sweep, every grid */
    double ms_total;         /* wall time of the call on the stream, ms */
    long long coarse_sweeps; /* sweeps of the coarsest-grid solves, summed over its visits */
    double history[64];      /* relative residual per finest-level check, in order (an
                                MG5_WARM solve's check of the initial guess comes first) */
} mg5_info;

/* ------------------------------------------------------------ utilities */

/* Library version, major * 100 + minor (1.00 = 100). */
int mg5_version(void);
const char *mg5_status_string(int status);
/* Number of CUDA kernel launches the library has enqueued in this process. */
long long mg5_kernel_launches(void);

/* Fill p with the defaults: nu1 = nu2 = 2, nu_coarse = 500, max_cycles = 100,
 * tol = 1e-10, precision MG5_FP64; alpha, s, h set to 0. */
int mg5_default_params(mg5_params *p);

/* Coefficients of Eq. (eomvarphi) for the normal-branch nDGP background
 * tuned to LCDM (Eq. dgpH), with beta(a) from Eq. (beta):
 *   beta = 1 + 2 H r_c (1 + Hdot / (3 H^2)),
 *   alpha = r_c^2 / (3 beta a^2)       [(Mpc/h)^2],
 *   s = Omega_m0 H0^2 / (beta a)       [(h/Mpc)^2],   c = 1, H0 = 1/2997.92458 h/Mpc.
 * a in (0, 1], omega_m0 in (0, 1], h0rc > 0.  Any output pointer may be NULL. */
int mg5_ndgp_coefficients(double a, double omega_m0, double h0rc, double *beta,
                          double *alpha, double *s);

/* Device bytes of scratch a solve of side N at `precision` allocates
 * (the HBM footprint used for admission). */
int mg5_workspace_bytes(int N, int precision, size_t *bytes);

/* ------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * scratch the context may hold (0 = no cap).  Returns MG5_E_ARG for a bad
 * device, MG5_E_CUDA if the device cannot be used. */
int mg5_create(mg5_ctx **ctx, int device, size_t hbm_budget_bytes);
int mg5_destroy(mg5_ctx *ctx);
const char *mg5_last_error(mg5_ctx *ctx);
/* Scratch bytes the context currently holds. */
size_t mg5_bytes_held(mg5_ctx *ctx);
/* Release every cached hierarchy (scratch) the context holds. */
int mg5_release(mg5_ctx *ctx);
/* How the context's solves wait for the GPU on the host (the per-cycle residual
 * read and the end of a solve): on = 1 sleeps on a blocking-sync event, on = 0
 * (default) spins, which answers sooner but holds a CPU core.  Many threads
 * solving at once on few cores (the server's workers) should sleep. */
int mg5_set_blocking_wait(mg5_ctx *ctx, int on);
/* on = 1: a solve (or batch, or MG5_GRAPH capture) first tunes the sweep schedule
 * of every grid side of its hierarchy that has no entry yet (mg5_autotune), before
 * any capture begins.  Default 0: untuned sides use the default schedule. */
int mg5_set_autotune(mg5_ctx *ctx, int on);
/* Bytes a solve of side N at `precision` would add to the context: 0 when its
 * hierarchy is already resident, else mg5_workspace_bytes. */
int mg5_cached_bytes(mg5_ctx *ctx, int N, int precision, size_t *extra);
/* Device bytes one cached MG5_GRAPH solve of side N holds (hierarchy, staging, graph state). */
int mg5_graph_workspace_bytes(int N, int with_grad, size_t *bytes);
/* Bytes an MG5_GRAPH solve of (N, *p, grad or not) would add: 0 when its graph is cached. */
int mg5_graph_cached_bytes(mg5_ctx *ctx, int N, const mg5_params *p, int with_grad, size_t *extra);

/* ------------------------------------------------------------ the hot path */

/*
 * Solve Eq. (eomvarphi) on the periodic N^3 domain grid (Sec. 3.1) and,
 * optionally, return the central-difference gradient (Sec. 3.2).
 *   delta : N^3 FP64, density contrast, read only.  Its mean is ignored
 *           (the mean of the source is absorbed by c).
 *   N     : even, >= 4; the grids halve while the half is even and >= 4; the
 *           coarsest grid must be at most 32 (else MG5_E_ARG).
 *   p     : parameters (alpha >= 0, s, h > 0, tol >= 0).
 *   flags : MG5_WARM (phi is the initial guess, else zero), MG5_HOST_IO, MG5_FMG, MG5_GRAPH.
 *   phi   : N^3 FP64, out: the solution with mean zero.
 *   grad  : 3 N^3 FP64 (gx, gy, gz blocks, SoA) or NULL; grad = d phi / dx_a.
 *           The fifth force on a particle is -grad / 2 (Eq. modpoisson).
 *   info  : may be NULL.
 * Synchronises `stream` once per V-cycle (the convergence test).
 * Returns MG5_OK, MG5_W_DISC_CLAMP, MG5_E_NOT_CONVERGED (phi = last
 * iterate), MG5_E_DIVERGED, MG5_E_NONFINITE, MG5_E_ARG, MG5_E_OOM, MG5_E_CUDA.
 */
int mg5_solve_fifth_force(mg5_ctx *ctx, const double *delta, int N, const mg5_params *p,
                          unsigned flags, double *phi, double *grad, mg5_info *info,
                          void *stream);

/*
 * Central-difference gradient (Sec. 3.2: the force is obtained by finite
 * differencing phi at cell centres):
 *   grad[a][cell] = (phi[cell + e_a] - phi[cell - e_a]) / (2 h).
 *   phi  : box of dims[0] x dims[1] x dims[2] FP64 (device).
 *   ghost: width of the ghost shell; the gradient is computed on the
 *          interior (dims - 2 ghost) and written SoA, 3 blocks of that size.
 *   periodic != 0: the box is a periodic cube (ghost must be 0).
 *   Non-periodic boxes need ghost >= 1.
 */
int mg5_force(mg5_ctx *ctx, const double *phi, const int dims[3], int ghost, double h,
              int periodic, double *grad, void *stream);

/*
 * Coarse-to-fine interpolation (Sec. 3.1: boundary values and initial guess
 * of a refinement; Sec. 3.2: the truncated fine-level phi).
 *   phi_coarse: Nc^3 periodic FP64 (device).
 *   o[3], pn[3]: the patch covers coarse cells [o, o + pn) on each axis
 *               (wrapping periodically); 0 <= o < Nc, 1 <= pn <= Nc.
 *   ghost:      fine ghost cells on every side (0..4).
 *   phi_fine:   out, (2 pn + 2 ghost) per axis, FP64 (device).
 * Fine local index I sits at coarse coordinate x = o + (I - ghost + 1/2)/2
 * (coarse centre m at m + 1/2) and gets the trilinear blend of the eight
 * nearest coarse centres (weights 3/4 and 1/4 per axis).
 */
int mg5_refine_interpolate(mg5_ctx *ctx, const double *phi_coarse, int Nc, const int o[3],
                           const int pn[3], int ghost, double *phi_fine, void *stream);

/*
 * Tricubic variant of mg5_refine_interpolate (an extension; the paper interpolates
 * without naming an order): per axis the 4-point Lagrange polynomial through the
 * coarse centres around the fine centre (weights (-7, 105, 35, -5)/128 a quarter
 * cell right of a centre, mirrored three quarters right), tensor product over the
 * axes; exact for cubic polynomials.  Same arguments as mg5_refine_interpolate;
 * Nc >= 4.
 */
int mg5_refine_interpolate_cubic(mg5_ctx *ctx, const double *phi_coarse, int Nc, const int o[3],
                                 const int pn[3], int ghost, double *phi_fine, void *stream);

/*
 * The same interpolation from a refinement's box instead of the periodic domain:
 * the next level of a nested hierarchy of refinements (Sec. 3.1, Fig. amr: each
 * refinement takes its boundary values and initial guess from its parent).
 *   box:    parent phi (device FP64), dims bd[3] including a ghost shell of pg
 *           cells; interior cell m of axis a is box index m + pg.
 *   o, pn:  the child covers parent interior cells [o, o + pn), inside the interior.
 *   ghost:  fine ghost cells on every side (0..4).
 * Every parent centre the trilinear stencil reaches must lie in the box (for
 * ghost = 1 a parent ghost shell of one cell suffices); MG5_E_ARG otherwise.
 */
int mg5_refine_interpolate_box(mg5_ctx *ctx, const double *box, const int bd[3], int pg,
                               const int o[3], const int pn[3], int ghost, double *phi_fine,
                               void *stream);

/*
 * Relax the refinement (the untruncated, "full" fine level of Sec. 3.2):
 * solve op(phi) = s delta_fine + compat_c on the interior pf[0] x pf[1] x
 * pf[2] of a box with a one-cell ghost shell whose values stay fixed
 * (Dirichlet boundary values from the coarse level, Sec. 3.1).
 *   delta_fine: pf[0]*pf[1]*pf[2] FP64 (device), the fine density contrast.
 *   p         : alpha, s, h (the FINE cell size), tol (relative to
 *               ||s delta_fine||_2), nu1, nu2, nu_coarse, max_cycles (V-cycle cap).
 *   compat_c  : the coarse solve's c (keeps the background consistent).
 *   phi_fine  : (pf + 2)^3 box (device): in, the initial guess and the fixed
 *               ghost shell (from mg5_refine_interpolate with ghost = 1);
 *               out, the relaxed interior (ghosts untouched).
 * Solved by FAS V-cycles on the patch (interior halved while every side is
 * even and the half >= 4; coarse ghost shells are means of the fine ghost
 * cells they cover, so coarse corrections vanish on the boundary).  Each pf
 * must be even and >= 2.  Synchronises `stream` once per V-cycle.
 */
int mg5_relax_patch(mg5_ctx *ctx, const double *delta_fine, const int pf[3],
                    const mg5_params *p, double compat_c, double *phi_fine,
                    mg5_info *info, void *stream);
/* mg5_relax_patch as ONE CUDA-graph launch: the context captures, per (pf, parameters), the
 * whole relaxation with its V-cycle loop as a device-controlled WHILE node (own hierarchy and
 * staging; compat_c is passed to the device on each call) and replays it: copy in, launch, copy
 * out, one synchronisation.  The same kernels as mg5_relax_patch, bit-identical results.  Needs
 * a patch hierarchy of two grids or more and nu1 + nu2 even (MG5_E_ARG otherwise). */
int mg5_relax_patch_graph(mg5_ctx *ctx, const double *delta_fine, const int pf[3],
                          const mg5_params *p, double compat_c, double *phi_fine,
                          mg5_info *info, void *stream);

/*
 * Position-dependent truncation (Sec. 3.3, the criterion proposed for screening
 * that does not follow the refinement): iterate a fine cell only while the
 * fifth force on its parent cell is still large.
 *
 * mg5_parent_force_mask builds the mask of a refinement from the parent level:
 *   grad_phi, grad_gr: gradients of phi and of the GR potential Psi_GR on the
 *            parent grid of dims pd, SoA 3 x pd[0] x pd[1] x pd[2] FP64 (device;
 *            the layout mg5_force writes, for the periodic domain or, with
 *            ghost = 1, for the interior of a refinement's box).
 *   periodic: != 0: the parent is the periodic domain (indices wrap;
 *            0 <= o < pd, 1 <= pn <= pd); 0: a refinement's interior
 *            (0 <= o, o + pn <= pd).
 *   o, pn:   the refinement covers parent cells [o, o + pn) per axis.
 *   theta:   threshold on |F5| / |F_GR|, F5 = grad(phi)/2 (Sec. 3.2), >= 0.
 *   mask:    out, (2 pn[0]) x (2 pn[1]) x (2 pn[2]) bytes (device), C order:
 *            1 where |F5| > theta |F_GR| at the cell's parent (compared without
 *            division: a parent with F_GR = 0 counts as large when F5 != 0),
 *            else 0.
 *   count:   if not NULL, out: the number of 1 entries (synchronises `stream`).
 *
 * mg5_relax_patch_masked is mg5_relax_patch iterating only the cells whose
 * mask byte is nonzero:
 *   mask: pf[0]*pf[1]*pf[2] bytes (device), interior-indexed like delta_fine.
 * Cells with mask 0 keep the values phi_fine holds on entry (the interpolated
 * parent phi) and act as fixed values for their iterated neighbours, like the
 * ghost shell.  Convergence: ||r|| <= tol ||s delta_fine|| with both norms over
 * the masked cells (an empty mask returns at once with 0 cycles).  The V-cycle
 * keeps a mask per grid: a coarse cell is relaxed only if all 8 of its children
 * are, residuals of unmasked cells restrict as zero and corrections reach masked
 * cells only.  When fewer than 10% of the cells are masked, masked sweeps alone
 * run first (the residual checked every 4, at most 64) and V-cycles take over only
 * if those have not converged; info->cycles counts V-cycles (0 when the sweeps
 * alone converged) and info->history every check.  Same other arguments, errors
 * and synchronisation as mg5_relax_patch (plus one synchronisation to read the
 * masked fraction); info->cell_updates counts every interior cell the sweeps visit.
 */
int mg5_parent_force_mask(mg5_ctx *ctx, const double *grad_phi, const double *grad_gr,
                          const int pd[3], int periodic, const int o[3], const int pn[3],
                          double theta, unsigned char *mask, long long *count, void *stream);
int mg5_relax_patch_masked(mg5_ctx *ctx, const double *delta_fine, const int pf[3],
                           const unsigned char *mask, const mg5_params *p, double compat_c,
                           double *phi_fine, mg5_info *info, void *stream);

/*
 * Solve many independent boxes in one call (batching).  Box i has side N[i],
 * density delta[i], parameters p[i], output phi[i] and, if grad is not NULL,
 * grad[i] (all device buffers, layouts as in mg5_solve_fifth_force; phi starts
 * from zero).  When every box is MG5_MIXED the whole batch is ONE CUDA graph
 * launch: a branch per box, each a WHILE loop of FP64 defect-correction steps
 * around FP32 V-cycles whose continuation a device kernel decides, so boxes
 * converge independently and overlap on the GPU with no host round trip.  The
 * graph and the per-box hierarchies stay resident and are reused while the
 * sizes, parameters and pointers are unchanged.  Otherwise the boxes are
 * solved one after another.  info: nbox entries or NULL.  Returns the worst
 * status over the boxes; synchronises `stream` once.
 */
int mg5_solve_batch(mg5_ctx *ctx, int nbox, const double *const *delta, const int *N,
                    const mg5_params *p, double *const *phi, double *const *grad, mg5_info *info,
                    void *stream);

/* ------------------------------------------------------------ autotuner
 * The smoother's schedule changes speed, not values: the two-pass sweep (a red
 * and a black kernel, `block` threads per block) or the fused plane-march
 * (one kernel, each CTA marching over `chunk` planes; 0 = enough CTAs for
 * several waves) apply the same cell update of Sec. 3.1 to the same snapshot.
 * The table is process-wide, keyed by (device, precision, grid side n); solves,
 * batch captures and MG5_GRAPH captures read it when they start (a captured
 * graph keeps the schedule it was captured with).  Defaults: FP64 two-pass with
 * 256 threads a block, or on grids too small to give each of the 152 SMs two such
 * blocks the multiple of 32 (at least 32) that does; the mixed mode's FP32 correction form as a column march where n is
 * a multiple of 32, else fused where n >= 32 and n % 4 == 0. */
#define MG5_SWEEP_TWO_PASS 0
#define MG5_SWEEP_FUSED    1
#define MG5_SWEEP_MARCH    2   /* MG5_MIXED's FP32 correction-form sweep as a column march
                                  (grid sides that are multiples of 32; others use the fused
                                  kernel); in MG5_FP64 it reads as MG5_SWEEP_FUSED */
typedef struct {
    int form;    /* MG5_SWEEP_TWO_PASS, MG5_SWEEP_FUSED or MG5_SWEEP_MARCH */
    int block;   /* threads per block of the two-pass kernels (32 .. 1024, a multiple of 32) */
    int chunk;   /* planes per CTA of the fused or march kernel (0 = automatic) */
    float ms;    /* the tuner's median time of one sweep (0 when set by hand) */
} mg5_schedule;
/* Time every candidate schedule (two-pass with 32/64/128/256/512 threads, fused with
 * 8/16/32 planes where it fits, and for MG5_MIXED the column march with automatic,
 * 16, 32, 64 or 128 planes where it fits) on a synthetic field of each grid side of the
 * hierarchy of N (coarsest excluded) on ctx's device and stream, and record the
 * fastest; sides already in the table are kept.  Synchronises `stream`; must not
 * run during a stream capture.  Allocates (and frees) 3-4 grids of the side. */
int mg5_autotune(mg5_ctx *ctx, int N, int precision, void *stream);
/* The schedule of (device, precision, n): MG5_OK if tuned or set, MG5_W_UNTUNED
 * with the default in *out otherwise. */
int mg5_schedule_get(int device, int precision, int n, mg5_schedule *out);
/* Set a schedule by hand (MG5_E_ARG for an invalid one). */
int mg5_schedule_set(int device, int precision, int n, const mg5_schedule *s);
/* Forget every entry (all devices). */
int mg5_tune_clear(void);
/* Write the table as JSON lines ({"gpu", "precision", "n", "form", "block",
 * "chunk", "ms"}), keyed by the GPU's name so a table tuned on one GPU model
 * loads on any GPU of that model. */
int mg5_tune_save(const char *path);
/* Apply the lines of a saved table whose GPU name matches a visible device:
 * returns how many entries were applied (>= 0), MG5_E_ARG for an unreadable
 * file or a malformed line (the well-formed lines are still applied). */
int mg5_tune_load(const char *path);

/* ------------------------------------------------------------ serving
 * A continuous-batching solve server: `slots` worker threads, each with its
 * own context (resident hierarchies) and CUDA stream.  Requests are admitted
 * in arrival order when a worker is free and the HBM the request adds fits
 * hbm_budget_bytes next to what all workers hold (0 = no cap); idle workers
 * drop cached hierarchies when an admission waits for memory.  Admitted solves
 * run concurrently, as replays of captured solves from a pool the workers share
 * (MG5_MIXED; MG5_FP64 with two grids or more and nu1 + nu2 even), else
 * host-driven on the worker's context.  Results are deterministic: the same
 * alone and in the mix. */
typedef struct mg5_server mg5_server;

typedef struct {
    const double *delta;     /* device, N^3, read until the request completes */
    int N;
    mg5_params params;
    double *phi;             /* device, N^3, written (zero start) */
    double *grad;            /* device, 3 N^3, or NULL */
    unsigned long long tag;  /* caller's identifier, echoed in the completion */
} mg5_request;

typedef struct {
    unsigned long long tag;
    int status;
    int pad;
    double t_submit, t_admit, t_done;   /* seconds on the server clock */
    mg5_info info;
} mg5_completion;

/* Start a server on `device` with `slots` workers (1..256) and an HBM cap (0 = none); *srv
 * receives the handle.  MG5_E_ARG for a bad device or slot count, MG5_E_CUDA if no device
 * can be queried; the workers start at once and wait for requests. */
int mg5_server_create(mg5_server **srv, int device, int slots, size_t hbm_budget_bytes);
/* Enqueue (thread-safe, non-blocking).  MG5_E_OOM if the request alone exceeds the budget
 * (a request that cannot fit even with every worker idle and empty completes with MG5_E_OOM). */
int mg5_server_submit(mg5_server *srv, const mg5_request *req);
/* Move up to max completions into out, waiting up to wait_ms for the first; returns the count. */
int mg5_server_poll(mg5_server *srv, mg5_completion *out, int max, int wait_ms);
/* Requests waiting for a worker and requests running (either pointer may be NULL). */
int mg5_server_pending(mg5_server *srv, int *queued, int *running);
/* Seconds since the server started: the clock of the completions' timestamps. */
double mg5_server_clock(mg5_server *srv);
/* Device bytes the server holds now (hierarchies, captured solves, staging). */
size_t mg5_server_bytes_held(mg5_server *srv);
/* Counters of a server since creation: captured graphs built, the seconds spent
 * building them (allocation + capture + instantiation), idle entries evicted for
 * memory, requests that ran host-driven because no graph could be built,
 * admissions that had to wait for memory, and requests completed. */
typedef struct {
    long long builds, evictions, fallbacks, memory_waits, completed;
    double build_seconds;
} mg5_server_stats;
/* Copy the counters into *out (thread-safe). */
int mg5_server_get_stats(mg5_server *s, mg5_server_stats *out);
/* Finish every queued request, stop the workers, free everything. */
int mg5_server_destroy(mg5_server *srv);

/* ------------------------------------------------------------ without allocation
 * For callers that cannot allocate device memory (code running inside a memory
 * pool or allocator it does not own, inside regions where an allocation would
 * synchronise the device or break an enclosing capture, or hosts that only
 * lend buffers they own).  This entry point has no counterpart in the paper:
 * it is the residual norm of the solve's stopping test (no context needed).
 *   out (device, 3 doubles) = mean r, ||r - mean r||_2, ||r||_2 for
 *   r = f + c - op(phi) on the periodic N^3 grid, op the operator of Eq. (eomvarphi)
 *   (phi, f: device, N^3 doubles, row-major, not modified; c, h, alpha as in the solve).
 * Each of at most 4096 blocks (256 threads, two cells a thread) reduces its
 * cells to (count, shift, sum and sum of squares of the deviations from the
 * shift), the shift one of its own residuals; the blocks are moved onto one shift
 * and summed in block order, so ||r - mean r|| keeps its accuracy when |mean r| is
 * far above the spread of r.  The block results live in a fixed
 * file-scope device array of 4096 x 32 bytes (128 KiB), held by every GPU that
 * loads the library until the process exits: N^3 may be at most
 * mg5_residual_norm_noalloc_max_cells() (2,097,152, i.e. N <= 128); larger grids
 * return MG5_E_TOO_LARGE.  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array,
 * so calls that overlap on the GPU (different streams, concurrent threads)
 * race; each call overwrites every slot it reads.  No cudaMalloc, no cudaFree. */
int mg5_residual_norm_noalloc(const double *phi, const double *f, double c, int N, double h,
                              double alpha, double *out, void *stream);
long long mg5_residual_norm_noalloc_max_cells(void);

/* ------------------------------------------------------------ tracing
 * Per-kernel-class device time, measured with CUDA events recorded on the
 * launching stream around each launch (off by default).  enable() also
 * clears the totals; read() synchronises the device, then copies up to n
 * totals (ms) and launch counts and returns the number of classes. */
int mg5_profile_enable(mg5_ctx *ctx, int on);
int mg5_profile_read(mg5_ctx *ctx, double *ms, long long *calls, int n);
/* Cells processed per class (fine-grid cells of each launch), for roofline arithmetic. */
int mg5_profile_units(mg5_ctx *ctx, double *units, int n);
const char *mg5_profile_name(int k);

/* ------------------------------------------------------------ single steps
 * Each runs one kernel of the hot path on device buffers, for testing the
 * steps one by one.  N is the periodic side (even); c is the compatibility
 * constant the step uses; f is the right-hand side (s delta on the domain grid). */

/* One snapshot red-black sweep (red = (i+j+k) even first; within a
 * half-sweep every value read is the value from before that half-sweep):
 * phi_out = sweep(phi_in).  phi_in and phi_out must not alias. */
int mg5_step_sweep(mg5_ctx *ctx, const double *phi_in, double *phi_out, const double *f,
                   double c, int N, double h, double alpha, void *stream);
/* Residual of the mixed mode's FP32 correction equation, r = f + c - (op(B + e) - op(B)),
 * restricted by 8-child means: ec = R e and rc = R r ((N/2)^3 floats each, device), with
 * stats (host, 2 doubles, may be NULL) = mean r and ||r - mean r||_2.  e, f, B: device,
 * N^3 floats.  variant 0: gather kernel; 1: column-march kernel (N a multiple of 32).
 * Both give the same ec and rc to the bit; the statistics agree to FP32 summation order.
 * Synchronises the stream. */
int mg5_step_resid_restrict_f32(mg5_ctx *ctx, const float *e, const float *f, const float *B,
                                double c, int N, double h, double alpha, int variant, float *ec,
                                float *rc, double *stats, void *stream);
/* The same sweep by the fused kernel (one read and one write of phi per cell). */
int mg5_step_sweep_fused(mg5_ctx *ctx, const double *phi_in, double *phi_out, const double *f,
                         double c, int N, double h, double alpha, void *stream);
/* FP32 sweep of the mixed-precision inner solve.  With B == NULL it is the
 * sweep above in FP32; with a base B it relaxes the correction e of
 * op(B + e) - op(B) = f + c (B fixed).  variant 0: two-pass kernel,
 * 1: fused kernel, 2: column-march kernel (needs B and N a multiple of 32).
 * Every variant computes the same values.  e_in and e_out must not alias. */
int mg5_step_sweep_f32(mg5_ctx *ctx, const float *e_in, float *e_out, const float *f,
                       const float *B, double c, int N, double h, double alpha, int variant,
                       void *stream);
/* out = op(phi) = L + alpha ((2/3) L^2 - Sigma) */
int mg5_step_operator(mg5_ctx *ctx, const double *phi, int N, double h, double alpha,
                      double *out, void *stream);
/* r = f + c - op(phi) */
int mg5_step_residual(mg5_ctx *ctx, const double *phi, const double *f, double c, int N,
                      double h, double alpha, double *r, void *stream);
/* coarse = mean of the 8 children of each coarse cell; N = fine side */
int mg5_step_restrict(mg5_ctx *ctx, const double *fine, int N, double *coarse, void *stream);
/* fine += cell-centred trilinear interpolation of coarse; Nc = coarse side */
int mg5_step_prolong_add(mg5_ctx *ctx, const double *coarse, int Nc, double *fine,
                         void *stream);

/* ------------------------------------------------------------ range-checked build
 * Debugging aids with no counterpart in the paper.  The library can be built with
 * -DMG5_BOUNDS (libmg5_bounds.so): every element a kernel reads or writes in global
 * memory is checked against the device allocations the library knows -- its own, each
 * registered at allocation, and the caller buffers noted with mg5_bounds_note -- and
 * shared-memory elements against the CTA's shared memory.  A violation does not fault:
 * the access is redirected to a scratch word (an asynchronous copy is skipped) and the
 * first violation per source file is recorded on the device.  The checks slow every
 * kernel by a large factor; results of a run without violations are those of the
 * ordinary build.  In the ordinary build these entry points do nothing. */
/* 1 in the range-checked build, 0 otherwise. */
int mg5_bounds_build(void);
/* Note the device allocation that contains p (a caller buffer) as readable and writable
 * by the kernels; MG5_E_ARG if p is not device memory.  MG5_OK (nothing done) in the
 * ordinary build. */
int mg5_bounds_note(const void *p);
/* Read and clear the recorded violations: 1 if any, with "file: line L: kind out of
 * range" for the first one written to msg (cap bytes, NUL-terminated), else 0.  Call it
 * after the device work has finished (a stream or device synchronisation). */
int mg5_bounds_check(char *msg, int cap);

#ifdef __cplusplus
}
#endif
#endif /* MG5_H */
