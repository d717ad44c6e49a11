/*
 * mg_oracle.c -- plain FP64 CPU oracle for the nDGP scalar-field solve.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library computes.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, table or constant with the CUDA library.
 *
 * Paper: Barreira, Bose & Li, "Speeding up N-body simulations of modified
 * gravity: Vainshtein screening models" (arXiv:1511.08200).
 *
 *   Eq. (eomvarphi)  lap(phi) + alpha [ (lap phi)^2 - (d_i d_j phi)^2 ] = s delta,
 *                    alpha = r_c^2 / (3 beta a^2),  s = 8 pi G a^2 rho_bar / (3 beta)
 *   Eq. (beta)       beta(a) = 1 + 2 H r_c (1 + Hdot / (3 H^2))
 *   Eq. (dgpH)       normal branch, background tuned to LCDM
 *   Eq. (eomgen-disc), Eq. (newton)  cell-by-cell iteration of T_ijk = 0
 *   Sec. 3.1         level-by-level solve: periodic domain grid first, V-cycles
 *   Sec. 3.2         truncation: fine phi = interpolant of coarse phi,
 *                    force by finite differencing phi at cell centres
 *
 * Readings taken where the paper is silent (each is listed in the design
 * notes): second-order central differences for the Hessian; the operator
 * split  (lap)^2 - (d d)^2 = (2/3) L^2 - Sigma  with Sigma independent of the
 * centre value; the exact quadratic root as the cell update (the fixed point
 * of the Newton update of Eq. newton); "snapshot" red-black ordering; a
 * compatibility constant c on the periodic grid; 8-child mean restriction and
 * cell-centred trilinear prolongation; FAS V-cycles.
 *
 * Layout: C order, index (i*N + j)*N + k, k fastest, i <-> x.
 * Nothing here is tuned: loops are written the way the definitions read.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* background coefficients: Eq. (dgpH) normal branch tuned to LCDM,    */
/* Eq. (beta), Eq. (eomvarphi)                                        */
/* ------------------------------------------------------------------ */

/* H0 in h/Mpc with c = 1: 100 km/s/Mpc divided by c in km/s. */
#define OR_H0_H_PER_MPC (100.0 / 299792.458)

/*
 * a: scale factor; om: Omega_m0; h0rc: H0 * r_c.
 * Outputs beta (Eq. beta), alpha = r_c^2/(3 beta a^2) in (Mpc/h)^2 and
 * s = Omega_m0 H0^2 / (beta a) in (h/Mpc)^2 (the source coefficient of
 * Eq. eomvarphi after writing 8 pi G rho_bar a^2 = 3 H0^2 Omega_m0 / a).
 */
void or_ndgp_coefficients(double a, double om, double h0rc, double *beta,
                          double *alpha, double *s)
{
    double E2 = om / (a * a * a) + (1.0 - om);        /* (H/H0)^2, LCDM */
    double E = sqrt(E2);
    /* Hdot / H^2 = (1/2) dln(H^2)/dln(a) for H = H(a(t)) */
    double hdot_over_h2 = -1.5 * om / (a * a * a) / E2;
    double b = 1.0 + 2.0 * E * h0rc * (1.0 + hdot_over_h2 / 3.0);
    double rc = h0rc / OR_H0_H_PER_MPC;
    *beta = b;
    *alpha = rc * rc / (3.0 * b * a * a);
    *s = om * OR_H0_H_PER_MPC * OR_H0_H_PER_MPC / (b * a);
}

/* ------------------------------------------------------------------ */
/* indexing                                                            */
/* ------------------------------------------------------------------ */

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* periodic cube of side n */
static double per(const double *a, int n, int i, int j, int k)
{
    return a[((size_t)wrap(i, n) * n + wrap(j, n)) * n + wrap(k, n)];
}

static size_t pidx(int n, int i, int j, int k)
{
    return ((size_t)i * n + j) * n + k;
}

/* A field accessor: either a periodic cube or a box without wrapping. */
typedef struct {
    const double *a;
    int d0, d1, d2;   /* box dims (ghosts included); cube: all = n */
    int periodic;
} or_field;

static double at(const or_field *f, int i, int j, int k)
{
    if (f->periodic)
        return per(f->a, f->d0, i, j, k);
    return f->a[((size_t)i * f->d1 + j) * f->d2 + k];
}

/* ------------------------------------------------------------------ */
/* discrete operator                                                   */
/* ------------------------------------------------------------------ */

/*
 * Second-order central-difference Hessian at (i,j,k):
 *   D_xx = (phi[i+1] + phi[i-1] - 2 phi) / h^2
 *   D_xy = (phi[i+1,j+1] - phi[i+1,j-1] - phi[i-1,j+1] + phi[i-1,j-1]) / (4 h^2)
 * H[0..5] = Dxx, Dyy, Dzz, Dxy, Dxz, Dyz.
 */
static void hessian(const or_field *f, int i, int j, int k, double h, double H[6])
{
    double c = at(f, i, j, k);
    double h2 = h * h;
    H[0] = (at(f, i + 1, j, k) + at(f, i - 1, j, k) - 2.0 * c) / h2;
    H[1] = (at(f, i, j + 1, k) + at(f, i, j - 1, k) - 2.0 * c) / h2;
    H[2] = (at(f, i, j, k + 1) + at(f, i, j, k - 1) - 2.0 * c) / h2;
    H[3] = (at(f, i + 1, j + 1, k) - at(f, i + 1, j - 1, k)
            - at(f, i - 1, j + 1, k) + at(f, i - 1, j - 1, k)) / (4.0 * h2);
    H[4] = (at(f, i + 1, j, k + 1) - at(f, i + 1, j, k - 1)
            - at(f, i - 1, j, k + 1) + at(f, i - 1, j, k - 1)) / (4.0 * h2);
    H[5] = (at(f, i, j + 1, k + 1) - at(f, i, j + 1, k - 1)
            - at(f, i, j - 1, k + 1) + at(f, i, j - 1, k - 1)) / (4.0 * h2);
}

/*
 * Left-hand side of Eq. (eomvarphi) at one cell, written as the definition:
 *   L + alpha [ L^2 - sum_ij (d_i d_j phi)^2 ],   L = Dxx + Dyy + Dzz,
 *   sum_ij (d_i d_j phi)^2 = Dxx^2 + Dyy^2 + Dzz^2 + 2 (Dxy^2 + Dxz^2 + Dyz^2).
 */
static double op_cell(const or_field *f, int i, int j, int k, double h, double alpha)
{
    double H[6];
    hessian(f, i, j, k, h, H);
    double L = H[0] + H[1] + H[2];
    double hh = H[0] * H[0] + H[1] * H[1] + H[2] * H[2]
              + 2.0 * (H[3] * H[3] + H[4] * H[4] + H[5] * H[5]);
    return L + alpha * (L * L - hh);
}

/* out[p] = op(phi)[p] on the periodic cube n^3 */
void or_operator(const double *phi, int n, double h, double alpha, double *out)
{
    or_field f = {phi, n, n, n, 1};
#pragma omp parallel for
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                out[pidx(n, i, j, k)] = op_cell(&f, i, j, k, h, alpha);
}

/* ------------------------------------------------------------------ */
/* the cell update                                                     */
/* ------------------------------------------------------------------ */

/*
 * Sigma = (d_i d_j phi)^2 - L^2/3 at (i,j,k), written through the
 * differences D_ii - D_jj (the centre value cancels) and the mixed D_ij
 * (the centre value is not used):
 *   Sigma = (1/3) sum_{i<j} (D_ii - D_jj)^2 + 2 sum_{i<j} D_ij^2.
 * Then (lap)^2 - (d d)^2 = (2/3) L^2 - Sigma.
 */
static double sigma_cell(const or_field *f, int i, int j, int k, double h)
{
    double h2 = h * h;
    double sx = at(f, i + 1, j, k) + at(f, i - 1, j, k);
    double sy = at(f, i, j + 1, k) + at(f, i, j - 1, k);
    double sz = at(f, i, j, k + 1) + at(f, i, j, k - 1);
    double dxy_d = (sx - sy) / h2, dxz_d = (sx - sz) / h2, dyz_d = (sy - sz) / h2;
    double H[6];
    hessian(f, i, j, k, h, H);
    return (dxy_d * dxy_d + dxz_d * dxz_d + dyz_d * dyz_d) / 3.0
         + 2.0 * (H[3] * H[3] + H[4] * H[4] + H[5] * H[5]);
}

static long long g_clamped; /* discriminant clamps, reset by the callers */
static long long g_cell_updates; /* bookkeeping only: cells relaxed, reset by or_solve */

/*
 * Solve  (2 alpha/3) L^2 + L - b = 0,  b = rhs + alpha Sigma,
 * for the root continuous with alpha -> 0 (L -> b), written in the
 * cancellation-free form L = 2 b / (1 + sqrt(1 + 8 alpha b / 3)).
 * A negative discriminant is clamped to zero and counted.
 */
static double physical_root(double b, double alpha)
{
    double disc = 1.0 + 8.0 * alpha * b / 3.0;
    if (disc < 0.0) {
        disc = 0.0;
#pragma omp atomic
        g_clamped++;
    }
    return 2.0 * b / (1.0 + sqrt(disc));
}

/*
 * New centre value at (i,j,k) with every neighbour held fixed: the exact
 * solution of T_ijk = 0 in the centre value (the fixed point of Eq. newton).
 *   L = (sum_faces phi - 6 phi_ijk) / h^2  =>  phi_ijk = (sum_faces - h^2 L) / 6.
 */
static double cell_update(const or_field *f, int i, int j, int k, double h,
                          double alpha, double rhs)
{
    double sf = at(f, i + 1, j, k) + at(f, i - 1, j, k) + at(f, i, j + 1, k)
              + at(f, i, j - 1, k) + at(f, i, j, k + 1) + at(f, i, j, k - 1);
    double b = rhs + alpha * sigma_cell(f, i, j, k, h);
    double L = physical_root(b, alpha);
    return (sf - h * h * L) / 6.0;
}

/* exported for the per-cell tests: value solving cell (i,j,k) of a periodic cube */
double or_cell_update(const double *phi, int n, int i, int j, int k, double h,
                      double alpha, double rhs)
{
    or_field f = {phi, n, n, n, 1};
    return cell_update(&f, i, j, k, h, alpha, rhs);
}

/* ------------------------------------------------------------------ */
/* snapshot red-black sweeps                                           */
/* ------------------------------------------------------------------ */

/*
 * One full sweep on the periodic cube n^3 (n even): red cells
 * ((i+j+k) even) first, then black.  Within a half-sweep every value that
 * is read comes from the state at the start of that half-sweep, so the
 * result does not depend on the visiting order; face neighbours have the
 * other colour and are therefore the latest values.  rhs = f + c.
 */
void or_sweep(double *phi, const double *f, double c, int n, double h, double alpha)
{
    size_t nc = (size_t)n * n * n;
    g_cell_updates += (long long)nc;
    double *snap = (double *)malloc(nc * sizeof(double));
    for (int colour = 0; colour < 2; ++colour) {
        memcpy(snap, phi, nc * sizeof(double));
        or_field sf = {snap, n, n, n, 1};
#pragma omp parallel for
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    if (((i + j + k) & 1) != colour)
                        continue;
                    size_t p = pidx(n, i, j, k);
                    phi[p] = cell_update(&sf, i, j, k, h, alpha, f[p] + c);
                }
    }
    free(snap);
}

/* r = f + c - op(phi) on the periodic cube */
void or_residual(const double *phi, const double *f, double c, int n, double h,
                 double alpha, double *r)
{
    or_operator(phi, n, h, alpha, r);
    size_t nc = (size_t)n * n * n;
    for (size_t p = 0; p < nc; ++p)
        r[p] = f[p] + c - r[p];
}

static double mean(const double *a, size_t n)
{
    double s = 0.0;
    for (size_t p = 0; p < n; ++p)
        s += a[p];
    return s / (double)n;
}

static double norm2(const double *a, size_t n)
{
    double s = 0.0;
    for (size_t p = 0; p < n; ++p)
        s += a[p] * a[p];
    return sqrt(s);
}

/* ------------------------------------------------------------------ */
/* grid transfers                                                      */
/* ------------------------------------------------------------------ */

/* coarse = mean of the 8 children; nf = fine side (even) */
void or_restrict(const double *fine, int nf, double *coarse)
{
    int nc = nf / 2;
    for (int I = 0; I < nc; ++I)
        for (int J = 0; J < nc; ++J)
            for (int K = 0; K < nc; ++K) {
                double s = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int d = 0; d < 2; ++d)
                            s += fine[pidx(nf, 2 * I + a, 2 * J + b, 2 * K + d)];
                coarse[pidx(nc, I, J, K)] = s / 8.0;
            }
}

/*
 * Cell-centred trilinear interpolation on a periodic coarse grid, evaluated
 * at the centre of fine cell (i,j,k): along each axis the fine centre lies
 * a quarter coarse cell from its parent's centre, so it takes 3/4 of the
 * parent and 1/4 of the parent's neighbour on that side.
 */
static double prolong_at(const double *coarse, int nc, int i, int j, int k)
{
    int P[3] = {i >> 1, j >> 1, k >> 1};
    int Q[3] = {(i & 1) ? P[0] + 1 : P[0] - 1, (j & 1) ? P[1] + 1 : P[1] - 1,
                (k & 1) ? P[2] + 1 : P[2] - 1};
    double v = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 2; ++d) {
                double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (d ? 0.25 : 0.75);
                v += w * per(coarse, nc, a ? Q[0] : P[0], b ? Q[1] : P[1], d ? Q[2] : P[2]);
            }
    return v;
}

/* fine += P(coarse) */
void or_prolong_add(const double *coarse, int nc, double *fine)
{
    int nf = 2 * nc;
    for (int i = 0; i < nf; ++i)
        for (int j = 0; j < nf; ++j)
            for (int k = 0; k < nf; ++k)
                fine[pidx(nf, i, j, k)] += prolong_at(coarse, nc, i, j, k);
}

/* ------------------------------------------------------------------ */
/* FAS V-cycle on the periodic hierarchy                               */
/* ------------------------------------------------------------------ */

#define OR_MAX_LEVELS 16

typedef struct {
    int n;
    double *v, *f, *v0, *r;
    double c;
} or_level;

/* number of levels: halve while the half is even and at least 4 */
int or_num_levels(int n)
{
    int L = 1;
    while ((n / 2) % 2 == 0 && n / 2 >= 4 && L < OR_MAX_LEVELS) {
        n /= 2;
        L++;
    }
    return L;
}

typedef struct {
    double alpha, s, h, tol;
    int nu1, nu2, nu_coarse, max_cycles;
} or_params;

typedef struct {
    int status;          /* 0 converged, 1 not converged, 2 diverged, 3 non-finite */
    int cycles;
    int levels;
    int coarsest_n;
    double rel_residual;
    double compat_c;
    double phi_mean_removed;
    long long clamped;
    long long cell_updates;   /* bookkeeping: cells relaxed, one per cell per sweep */
    double history[128];
} or_info;

/* coarse-grid relative reduction that ends the coarsest solve */
#define OR_COARSE_RTOL 1e-3

/*
 * Coarsest solve: before each sweep recompute c = mean(op(v) - f) and the
 * residual norm; stop once the norm is at most OR_COARSE_RTOL times the
 * first one, or after nu_coarse sweeps.
 */
static void coarsest(or_level *lv, double h, double alpha, int nu_coarse)
{
    size_t nc = (size_t)lv->n * lv->n * lv->n;
    double r0 = -1.0;
    for (int it = 0; it < nu_coarse; ++it) {
        or_residual(lv->v, lv->f, 0.0, lv->n, h, alpha, lv->r);
        double m = mean(lv->r, nc);              /* r = f - op(v) */
        lv->c = -m;                              /* c = mean(op(v) - f) */
        double s2 = 0.0;
        for (size_t p = 0; p < nc; ++p)
            s2 += (lv->r[p] - m) * (lv->r[p] - m);
        double rn = sqrt(s2);
        if (r0 < 0.0)
            r0 = rn;
        if (rn <= OR_COARSE_RTOL * r0)
            break;
        or_sweep(lv->v, lv->f, lv->c, lv->n, h, alpha);
    }
}

static void vcycle(or_level *lv, int l, int nlev, double h, double alpha,
                   const or_params *p)
{
    or_level *L = &lv[l];
    size_t nc = (size_t)L->n * L->n * L->n;
    if (l == nlev - 1) {
        coarsest(L, h, alpha, p->nu_coarse);
        return;
    }
    for (int s = 0; s < p->nu1; ++s)
        or_sweep(L->v, L->f, L->c, L->n, h, alpha);
    /* residual with the mean projected out; the projection updates c */
    or_residual(L->v, L->f, L->c, L->n, h, alpha, L->r);
    double m = mean(L->r, nc);
    L->c -= m;
    for (size_t q = 0; q < nc; ++q)
        L->r[q] -= m;
    or_level *C = &lv[l + 1];
    size_t ncc = (size_t)C->n * C->n * C->n;
    double hc = 2.0 * h;
    or_restrict(L->v, L->n, C->v);
    memcpy(C->v0, C->v, ncc * sizeof(double));
    or_restrict(L->r, L->n, C->r);
    or_operator(C->v, C->n, hc, alpha, C->f);
    for (size_t q = 0; q < ncc; ++q)
        C->f[q] += C->r[q];
    C->c = 0.0;
    vcycle(lv, l + 1, nlev, hc, alpha, p);
    for (size_t q = 0; q < ncc; ++q)
        C->v[q] -= C->v0[q];
    or_prolong_add(C->v, C->n, L->v);
    L->c += C->c;
    for (int s = 0; s < p->nu2; ++s)
        or_sweep(L->v, L->f, L->c, L->n, h, alpha);
}

/*
 * Solve op(phi) = s delta + c on the periodic cube n^3 with mean(phi) = 0
 * (Eq. eomvarphi on the domain grid, Sec. 3.1).  phi holds the initial guess
 * on entry (zero, or the previous solution) and the solution on exit.
 * Each cycle: nu1 sweeps, residual (the stopping test is made here, on the
 * iterate just smoothed), coarse-grid correction, nu2 sweeps.
 * Stops when ||r - mean r||_2 <= tol ||s delta||_2.
 */
int or_solve(const double *delta, int n, const or_params *p, double *phi, or_info *info)
{
    int nlev = or_num_levels(n);
    or_level lv[OR_MAX_LEVELS];
    int m = n;
    for (int l = 0; l < nlev; ++l) {
        size_t nc = (size_t)m * m * m;
        lv[l].n = m;
        lv[l].v = l == 0 ? phi : (double *)calloc(nc, sizeof(double));
        lv[l].f = (double *)calloc(nc, sizeof(double));
        lv[l].v0 = (double *)calloc(nc, sizeof(double));
        lv[l].r = (double *)calloc(nc, sizeof(double));
        lv[l].c = 0.0;
        m /= 2;
    }
    size_t n3 = (size_t)n * n * n;
    for (size_t q = 0; q < n3; ++q)
        lv[0].f[q] = p->s * delta[q];
    double fnorm = norm2(lv[0].f, n3);
    g_clamped = 0;
    g_cell_updates = 0;
    memset(info, 0, sizeof(*info));
    info->levels = nlev;
    info->coarsest_n = lv[nlev - 1].n;
    info->status = 1;
    double best = INFINITY;
    for (int cyc = 0;; ++cyc) {
        or_level *L = &lv[0];
        double rel;
        if (nlev == 1) {
            coarsest(L, p->h, p->alpha, p->nu_coarse);
            or_residual(L->v, L->f, L->c, n, p->h, p->alpha, L->r);
            double mm = mean(L->r, n3);
            L->c -= mm;
            for (size_t q = 0; q < n3; ++q)
                L->r[q] -= mm;
            rel = fnorm > 0.0 ? norm2(L->r, n3) / fnorm : norm2(L->r, n3);
        } else {
            for (int s = 0; s < p->nu1; ++s)
                or_sweep(L->v, L->f, L->c, n, p->h, p->alpha);
            or_residual(L->v, L->f, L->c, n, p->h, p->alpha, L->r);
            double mm = mean(L->r, n3);
            L->c -= mm;
            for (size_t q = 0; q < n3; ++q)
                L->r[q] -= mm;
            rel = fnorm > 0.0 ? norm2(L->r, n3) / fnorm : norm2(L->r, n3);
        }
        if (cyc < 128)
            info->history[cyc] = rel;
        info->cycles = cyc;
        info->rel_residual = rel;
        if (!isfinite(rel)) {
            info->status = 3;
            break;
        }
        if (rel <= p->tol) {
            info->status = 0;
            break;
        }
        if (rel < best)
            best = rel;
        if (cyc >= 3 && rel > 10.0 * best) {
            info->status = 2;
            break;
        }
        if (cyc >= p->max_cycles) {
            info->status = 1;
            break;
        }
        if (nlev == 1)
            continue;
        /* coarse-grid correction and post-smoothing of this cycle */
        or_level *C = &lv[1];
        size_t ncc = (size_t)C->n * C->n * C->n;
        double hc = 2.0 * p->h;
        or_restrict(L->v, n, C->v);
        memcpy(C->v0, C->v, ncc * sizeof(double));
        or_restrict(L->r, n, C->r);
        or_operator(C->v, C->n, hc, p->alpha, C->f);
        for (size_t q = 0; q < ncc; ++q)
            C->f[q] += C->r[q];
        C->c = 0.0;
        vcycle(lv, 1, nlev, hc, p->alpha, p);
        for (size_t q = 0; q < ncc; ++q)
            C->v[q] -= C->v0[q];
        or_prolong_add(C->v, C->n, L->v);
        L->c += C->c;
        for (int s = 0; s < p->nu2; ++s)
            or_sweep(L->v, L->f, L->c, n, p->h, p->alpha);
    }
    double pm = mean(phi, n3);
    for (size_t q = 0; q < n3; ++q)
        phi[q] -= pm;
    info->phi_mean_removed = pm;
    info->compat_c = lv[0].c;
    info->clamped = g_clamped;
    info->cell_updates = g_cell_updates;
    for (int l = 0; l < nlev; ++l) {
        if (l > 0)
            free(lv[l].v);
        free(lv[l].f);
        free(lv[l].v0);
        free(lv[l].r);
    }
    return info->status;
}

/* ------------------------------------------------------------------ */
/* force, Sec. 3.2: central differences of phi at cell centres         */
/* ------------------------------------------------------------------ */

/*
 * grad[a][cell] = (phi[cell + e_a] - phi[cell - e_a]) / (2h), written SoA,
 * over the interior of a box of dims d[3] (ghost width g on every side), or
 * over the whole periodic cube when periodic != 0 (then g must be 0).
 */
void or_force(const double *phi, const int d[3], int g, double h, int periodic,
              double *grad)
{
    or_field f = {phi, d[0], d[1], d[2], periodic};
    int n0 = d[0] - 2 * g, n1 = d[1] - 2 * g, n2 = d[2] - 2 * g;
    size_t ni = (size_t)n0 * n1 * n2;
    for (int i = 0; i < n0; ++i)
        for (int j = 0; j < n1; ++j)
            for (int k = 0; k < n2; ++k) {
                int I = i + g, J = j + g, K = k + g;
                size_t q = ((size_t)i * n1 + j) * n2 + k;
                grad[q] = (at(&f, I + 1, J, K) - at(&f, I - 1, J, K)) / (2.0 * h);
                grad[ni + q] = (at(&f, I, J + 1, K) - at(&f, I, J - 1, K)) / (2.0 * h);
                grad[2 * ni + q] = (at(&f, I, J, K + 1) - at(&f, I, J, K - 1)) / (2.0 * h);
            }
}

/* ------------------------------------------------------------------ */
/* coarse -> fine interpolation (Sec. 3.1 boundary values and initial  */
/* guess of a refinement; Sec. 3.2 truncated fine phi)                 */
/* ------------------------------------------------------------------ */

/*
 * The fine patch covers coarse cells [o, o + pn) on each axis, refined 2x,
 * plus a ghost shell of g fine cells; its dims are 2 pn + 2 g.  Fine local
 * index I (0 .. 2pn + 2g - 1) has its centre at coarse coordinate
 *   x = o + (I - g + 1/2) / 2,
 * with coarse centre m at m + 1/2.  The value is the trilinear blend of the
 * eight surrounding coarse centres, wrapped periodically.
 */
void or_refine_interpolate(const double *phic, int nc, const int o[3], const int pn[3],
                           int g, double *fine)
{
    int d[3];
    for (int a = 0; a < 3; ++a)
        d[a] = 2 * pn[a] + 2 * g;
    for (int I = 0; I < d[0]; ++I)
        for (int J = 0; J < d[1]; ++J)
            for (int K = 0; K < d[2]; ++K) {
                int loc[3] = {I, J, K};
                int i0[3];
                double w[3];
                for (int a = 0; a < 3; ++a) {
                    double x = o[a] + (loc[a] - g + 0.5) / 2.0;
                    double t = x - 0.5;
                    i0[a] = (int)floor(t);
                    w[a] = t - i0[a];
                }
                double v = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        for (int c = 0; c < 2; ++c) {
                            double wt = (a ? w[0] : 1.0 - w[0]) * (b ? w[1] : 1.0 - w[1])
                                      * (c ? w[2] : 1.0 - w[2]);
                            v += wt * per(phic, nc, i0[0] + a, i0[1] + b, i0[2] + c);
                        }
                fine[((size_t)I * d[1] + J) * d[2] + K] = v;
            }
}

/*
 * Higher-order variant of the same interpolation (an extension, not in the
 * paper): per axis the 4-point Lagrange polynomial through the coarse centres
 * i0 - 1 .. i0 + 2 around the fine centre, evaluated at its offset w from i0;
 * the tensor product of the three axes.  Reproduces cubic polynomials.
 */
static double lagrange4(int k, double w)
{
    switch (k) {
    case 0: return -w * (w - 1.0) * (w - 2.0) / 6.0;
    case 1: return (w + 1.0) * (w - 1.0) * (w - 2.0) / 2.0;
    case 2: return -(w + 1.0) * w * (w - 2.0) / 2.0;
    default: return (w + 1.0) * w * (w - 1.0) / 6.0;
    }
}

void or_refine_cubic(const double *phic, int nc, const int o[3], const int pn[3], int g,
                     double *fine)
{
    int d[3];
    for (int a = 0; a < 3; ++a)
        d[a] = 2 * pn[a] + 2 * g;
    for (int I = 0; I < d[0]; ++I)
        for (int J = 0; J < d[1]; ++J)
            for (int K = 0; K < d[2]; ++K) {
                int loc[3] = {I, J, K};
                int i0[3];
                double w[3];
                for (int a = 0; a < 3; ++a) {
                    double t = o[a] + (loc[a] - g + 0.5) / 2.0 - 0.5;
                    i0[a] = (int)floor(t);
                    w[a] = t - i0[a];
                }
                double v = 0.0;
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b)
                        for (int c = 0; c < 4; ++c)
                            v += lagrange4(a, w[0]) * lagrange4(b, w[1]) * lagrange4(c, w[2]) *
                                 per(phic, nc, i0[0] - 1 + a, i0[1] - 1 + b, i0[2] - 1 + c);
                fine[((size_t)I * d[1] + J) * d[2] + K] = v;
            }
}

/* ------------------------------------------------------------------ */
/* patch relaxation with fixed (Dirichlet) ghost values (Sec. 3.1)      */
/* ------------------------------------------------------------------ */

/*
 * One snapshot red-black sweep on the interior of a box with a ghost shell
 * of width 1: dims d = pf + 2.  Colour is the parity of the interior index.
 * mask (interior-indexed, may be NULL = every cell): cells with mask 0 are
 * not relaxed and keep their values (Sec. 3.3: iterations on some cells of a
 * level only).
 */
static void patch_sweep(double *phi, const double *f, double c, const int d[3], double h,
                        double alpha, const unsigned char *mask)
{
    size_t nc = (size_t)d[0] * d[1] * d[2];
    double *snap = (double *)malloc(nc * sizeof(double));
    for (int colour = 0; colour < 2; ++colour) {
        memcpy(snap, phi, nc * sizeof(double));
        or_field sf = {snap, d[0], d[1], d[2], 0};
#pragma omp parallel for
        for (int i = 1; i < d[0] - 1; ++i)
            for (int j = 1; j < d[1] - 1; ++j)
                for (int k = 1; k < d[2] - 1; ++k) {
                    if (((i - 1 + j - 1 + k - 1) & 1) != colour)
                        continue;
                    size_t bq = ((size_t)i * d[1] + j) * d[2] + k;
                    size_t iq = ((size_t)(i - 1) * (d[1] - 2) + (j - 1)) * (d[2] - 2) + (k - 1);
                    if (mask && !mask[iq])
                        continue;
                    phi[bq] = cell_update(&sf, i, j, k, h, alpha, f[iq] + c);
                }
    }
    free(snap);
}

/* r = f + c - op(phi) over the interior (interior-indexed output) */
void or_patch_residual(const double *phi, const double *f, double c, const int pf[3],
                       double h, double alpha, double *r)
{
    int d[3] = {pf[0] + 2, pf[1] + 2, pf[2] + 2};
    or_field sf = {phi, d[0], d[1], d[2], 0};
    for (int i = 0; i < pf[0]; ++i)
        for (int j = 0; j < pf[1]; ++j)
            for (int k = 0; k < pf[2]; ++k) {
                size_t iq = ((size_t)i * pf[1] + j) * pf[2] + k;
                r[iq] = f[iq] + c - op_cell(&sf, i + 1, j + 1, k + 1, h, alpha);
            }
}

/*
 * Relax op(phi) = s delta_f + c on the interior pf[0] x pf[1] x pf[2] of a
 * fine patch whose ghost shell (width 1) holds fixed values.  phi has dims
 * pf + 2 and holds the interpolated initial guess and ghosts on entry.
 * Sweeps until ||r||_2 <= tol ||s delta_f||_2 (checked every `check` sweeps)
 * or max_sweeps.  Returns the number of sweeps made.
 */
int or_relax_patch(const double *delta_f, const int pf[3], double alpha, double s,
                   double h, double c, double tol, int max_sweeps, int check,
                   double *phi, double *rel_out)
{
    int d[3] = {pf[0] + 2, pf[1] + 2, pf[2] + 2};
    size_t ni = (size_t)pf[0] * pf[1] * pf[2];
    double *f = (double *)malloc(ni * sizeof(double));
    double *r = (double *)malloc(ni * sizeof(double));
    for (size_t q = 0; q < ni; ++q)
        f[q] = s * delta_f[q];
    double fn = norm2(f, ni);
    int sweeps = 0;
    double rel = INFINITY;
    g_clamped = 0;
    for (;;) {
        or_patch_residual(phi, f, c, pf, h, alpha, r);
        rel = fn > 0.0 ? norm2(r, ni) / fn : norm2(r, ni);
        if (rel <= tol || sweeps >= max_sweeps || !isfinite(rel))
            break;
        for (int q = 0; q < check && sweeps < max_sweeps; ++q, ++sweeps)
            patch_sweep(phi, f, c, d, h, alpha, NULL);
    }
    if (rel_out)
        *rel_out = rel;
    free(f);
    free(r);
    return sweeps;
}

/* one patch sweep, exported for the per-step tests */
void or_patch_sweep(double *phi, const double *f, double c, const int pf[3], double h,
                    double alpha)
{
    int d[3] = {pf[0] + 2, pf[1] + 2, pf[2] + 2};
    patch_sweep(phi, f, c, d, h, alpha, NULL);
}

/* ------------------------------------------------------------------ */
/* position-dependent truncation (Sec. 3.3)                            */
/* ------------------------------------------------------------------ */

/*
 * The parent criterion of Sec. 3.3: a fine cell of a refinement is iterated
 * only while the fifth force on its parent (the coarse cell that was refined)
 * is still large compared with normal gravity.  F5 = grad(phi)/2 (Sec. 3.2),
 * F_GR = grad(Psi_GR); both given on the parent grid as SoA, 3 blocks of
 * pd[0] x pd[1] x pd[2] (or_force layout).  The parent is the periodic domain
 * (periodic != 0: indices wrap) or a refinement's interior (periodic = 0).
 * The refinement covers parent cells [o, o + pn) per axis; fine interior cell
 * (I, J, K) of the (2 pn) interior has parent (o + I/2, o + J/2, o + K/2).
 *   mask = 1  where |F5| > theta |F_GR| at the parent, else 0
 * (no division: a parent with F_GR = 0 is iterated if F5 != 0).
 */
void or_parent_force_mask(const double *grad_phi, const double *grad_gr, const int pd[3],
                          int periodic, const int o[3], const int pn[3], double theta,
                          unsigned char *mask)
{
    size_t n3 = (size_t)pd[0] * pd[1] * pd[2];
    int P[3] = {2 * pn[0], 2 * pn[1], 2 * pn[2]};
    for (int I = 0; I < P[0]; ++I)
        for (int J = 0; J < P[1]; ++J)
            for (int K = 0; K < P[2]; ++K) {
                int c[3] = {o[0] + I / 2, o[1] + J / 2, o[2] + K / 2};
                if (periodic)
                    for (int a = 0; a < 3; ++a)
                        c[a] = wrap(c[a], pd[a]);
                size_t pc = ((size_t)c[0] * pd[1] + c[1]) * pd[2] + c[2];
                double f5 = 0.0, fg = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double x = 0.5 * grad_phi[a * n3 + pc], y = grad_gr[a * n3 + pc];
                    f5 += x * x;
                    fg += y * y;
                }
                mask[((size_t)I * P[1] + J) * P[2] + K] = sqrt(f5) > theta * sqrt(fg) ? 1 : 0;
            }
}

/*
 * or_relax_patch with iterations on the cells of `mask` only (Sec. 3.3): the
 * cells with mask 0 keep their entry values (the interpolated coarse phi) and
 * act, like the ghost shell, as fixed values for their iterated neighbours.
 * The residual and the source norm are taken over the iterated cells:
 * sweeps until ||r||_mask <= tol ||s delta_f||_mask.  Returns the sweeps made.
 */
int or_relax_patch_masked(const double *delta_f, const int pf[3], double alpha, double s,
                          double h, double c, const unsigned char *mask, double tol,
                          int max_sweeps, int check, double *phi, double *rel_out)
{
    int d[3] = {pf[0] + 2, pf[1] + 2, pf[2] + 2};
    size_t ni = (size_t)pf[0] * pf[1] * pf[2];
    double *f = (double *)malloc(ni * sizeof(double));
    double *fm = (double *)malloc(ni * sizeof(double));
    double *r = (double *)malloc(ni * sizeof(double));
    for (size_t q = 0; q < ni; ++q) {
        f[q] = s * delta_f[q];
        fm[q] = mask[q] ? f[q] : 0.0;
    }
    double fn = norm2(fm, ni);
    int sweeps = 0;
    double rel = INFINITY;
    g_clamped = 0;
    for (;;) {
        or_patch_residual(phi, f, c, pf, h, alpha, r);
        for (size_t q = 0; q < ni; ++q)
            if (!mask[q])
                r[q] = 0.0;
        rel = fn > 0.0 ? norm2(r, ni) / fn : norm2(r, ni);
        if (rel <= tol || sweeps >= max_sweeps || !isfinite(rel))
            break;
        for (int q = 0; q < check && sweeps < max_sweeps; ++q, ++sweeps)
            patch_sweep(phi, f, c, d, h, alpha, mask);
    }
    if (rel_out)
        *rel_out = rel;
    free(f);
    free(fm);
    free(r);
    return sweeps;
}

long long or_clamped(void)
{
    return g_clamped;
}
