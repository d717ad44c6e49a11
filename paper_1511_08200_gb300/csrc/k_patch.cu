// k_patch.cu -- kernels of the Dirichlet FAS multigrid on a refinement patch.
//
// A refinement of Sec. 3.1 has boundary values fixed by interpolation from
// the coarser level: the patch is a box whose one-cell ghost shell holds
// those values and is never relaxed.  Its FAS hierarchy halves the interior
// (8-child mean for the iterate and the residual); the coarse boxes carry a
// ghost shell too.  The saved coarse copy v0 keeps the ghosts filled once per
// solve by averaging the fine ghost cells each coarse ghost cell covers; the
// coarse iterate's ghosts follow the boundary condition of the correction
// below, and the prolongation reads the correction across the boundary.
//
// The fine problem fixes its correction to zero at the fine ghost centres,
// half a fine cell outside the first interior centre.  A coarse ghost centre
// lies farther out, so on coarse grid l the ghost value of the iterate is
// refreshed as  v0(g) + w^m (v(a) - v0(a)),  a the nearest interior cell, m the
// number of axes on which g lies outside, w = -(2^(l-1) - 1/2) / (2^(l-1) + 1/2)
// (-1/3 on grid 1): the linear extrapolation that puts the zero of the
// correction at the fine ghost centre.  The prolongation then gives the first
// fine cell 2/3 of its parent's correction, the linear interpolant between the
// boundary and the parent centre.
//
// Box layout: interior dims (p0, p1, p2), box dims (p + 2), interior index
// i <-> box index i + 1, C order.  Right-hand sides are interior-indexed.
#include "mg5_fin.cuh"

namespace mg5 {

__device__ __forceinline__ long long bidx(int i, int j, int k, int d1, int d2)
{
    return ((long long)i * d1 + j) * d2 + k;
}

// The ghosts of a coarse box anchored at its interior cell (I, J, K) (0-based), reset to v0's
// fixed values: right after the restriction v = v0 in the interior, so the boundary condition
// v0(g) + w^m (v(a) - v0(a)) of every ghost is v0(g) itself.  The restriction does this for the
// cells it writes, instead of a refresh launch over the box before the coarse right-hand side.
__device__ __forceinline__ void reset_anchored_ghosts(double *__restrict__ vc,
                                                      const double *__restrict__ v0c, int I, int J,
                                                      int K, int q0, int q1, int q2)
{
    const bool li = I == 0, hi = I == q0 - 1, lj = J == 0, hj = J == q1 - 1, lk = K == 0,
               hk = K == q2 - 1;
    if (!(li | hi | lj | hj | lk | hk))
        return;
    const int d1 = q1 + 2, d2 = q2 + 2;
    const int Iv[3] = {I + 1, 0, q0 + 1}, Jv[3] = {J + 1, 0, q1 + 1}, Kv[3] = {K + 1, 0, q2 + 1};
    const bool oi[3] = {true, li, hi}, oj[3] = {true, lj, hj}, ok[3] = {true, lk, hk};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if ((a | b | c) == 0 || !(oi[a] && oj[b] && ok[c]))
                    continue;
                const long long g = bidx(Iv[a], Jv[b], Kv[c], d1, d2);
                MG5_AT(vc, g) = MG5_AT(v0c, g);
            }
}

// residual of the 8 interior children of each coarse interior cell, restricted
// with v onto the coarse box interior (vc and v0c, vc's ghosts reset to v0c's) and into fc
// (interior-indexed).
// MASKED: the residual of a child with mask 0 (not iterated) counts as zero.
template <bool MASKED>
__global__ void k_pbox_resid_restrict(const double *__restrict__ v, const double *__restrict__ f,
                                      int p0, int p1, int p2, CoefT<double> cf,
                                      double *__restrict__ vc, double *__restrict__ v0c,
                                      double *__restrict__ fc, double2 *__restrict__ partials,
                                      const unsigned char *__restrict__ mask, Fin fin)
{
    const int q0 = p0 >> 1, q1 = p1 >> 1, q2 = p2 >> 1;
    const long long total = (long long)q0 * q1 * q2;
    double2 acc = make_double2(0.0, 0.0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int K = (int)(t % q2);
        const long long q = t / q2;
        const int J = (int)(q % q1), I = (int)(q / q1);
        double sv = 0.0, sr = 0.0;
        for (int ch = 0; ch < 8; ++ch) {
            const int i = 2 * I + (ch >> 2), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch & 1);
            const Rows r = box_rows(p1 + 2, p2 + 2, i + 1, j + 1);
            St<double> s;
            gather(v, v, r, k + 1, k + 2, k, s);
            const long long fi = ((long long)i * p1 + j) * p2 + k;
            const double res = (MASKED && !MG5_AT(mask, fi)) ? 0.0 : cell_residual(s, MG5_AT(f, fi), cf);
            sv += s.c;
            sr += res;
            acc.x += res;
            acc.y += res * res;
        }
        const long long cb = bidx(I + 1, J + 1, K + 1, q1 + 2, q2 + 2);
        MG5_AT(vc, cb) = 0.125 * sv;
        MG5_AT(v0c, cb) = 0.125 * sv;
        MG5_AT(fc, t) = 0.125 * sr;
        reset_anchored_ghosts(vc, v0c, I, J, K, q0, q1, q2);
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = acc;
    if (fin.ls)
        finalize_if_last(partials, fin);
}

// The same with a thread per fine cell, for the patch's coarse grids (up to kChildMaxFine fine
// cells; above that the FP64 pipe, not the chain, sets the time): eight consecutive lanes
// hold the eight children of one coarse cell (child ch = lane & 7, offsets ch >> 2,
// (ch >> 1) & 1, ch & 1) and sum their centres and residuals by three butterfly shuffles,
// ((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7)): one FP64 residual a thread instead of a
// chain of eight, which set the time of the patch's coarse grids (FP64 runs at 2 lanes a clock
// per SM on GB300).  The loop runs over whole warps, so every lane reaches the shuffles.
template <bool MASKED>
__global__ void k_pbox_resid_restrict_child(const double *__restrict__ v,
                                            const double *__restrict__ f, int p0, int p1, int p2,
                                            CoefT<double> cf, double *__restrict__ vc,
                                            double *__restrict__ v0c, double *__restrict__ fc,
                                            double2 *__restrict__ partials,
                                            const unsigned char *__restrict__ mask, Fin fin)
{
    const int q0 = p0 >> 1, q1 = p1 >> 1, q2 = p2 >> 1;
    const long long total = (long long)q0 * q1 * q2;
    const int lane = threadIdx.x & 31, ch = lane & 7;
    const long long stride = (long long)gridDim.x * blockDim.x / 8;   // coarse cells a pass
    double2 acc = make_double2(0.0, 0.0);
    for (long long t0 = ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / 8; t0 < total;
         t0 += stride) {
        const long long t = t0 + (lane >> 3);
        const bool live = t < total;
        double cv = 0.0, res = 0.0;
        int I = 0, J = 0, K = 0;
        if (live) {
            K = (int)(t % q2);
            const long long q = t / q2;
            J = (int)(q % q1);
            I = (int)(q / q1);
            const int i = 2 * I + (ch >> 2), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch & 1);
            const Rows r = box_rows(p1 + 2, p2 + 2, i + 1, j + 1);
            St<double> s;
            gather(v, v, r, k + 1, k + 2, k, s);
            const long long fi = ((long long)i * p1 + j) * p2 + k;
            res = (MASKED && !MG5_AT(mask, fi)) ? 0.0 : cell_residual(s, MG5_AT(f, fi), cf);
            cv = s.c;
            acc.x += res;
            acc.y += res * res;
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            cv += __shfl_xor_sync(0xffffffffu, cv, o);
            res += __shfl_xor_sync(0xffffffffu, res, o);
        }
        if (live && ch == 0) {
            const long long cb = bidx(I + 1, J + 1, K + 1, q1 + 2, q2 + 2);
            MG5_AT(vc, cb) = 0.125 * cv;
            MG5_AT(v0c, cb) = 0.125 * cv;
            MG5_AT(fc, t) = 0.125 * res;
            reset_anchored_ghosts(vc, v0c, I, J, K, q0, q1, q2);
        }
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = acc;
    if (fin.ls)
        finalize_if_last(partials, fin);
}

// fc = op(vc) + fc on the coarse interior (fc holds the restricted residual)
__global__ void k_pbox_coarse_rhs(const double *__restrict__ vc, double *__restrict__ fc, int q0,
                                  int q1, int q2, CoefT<double> cf)
{
    const long long total = (long long)q0 * q1 * q2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int k = (int)(t % q2);
    const long long q = t / q2;
    const int j = (int)(q % q1), i = (int)(q / q1);
    const Rows r = box_rows(q1 + 2, q2 + 2, i + 1, j + 1);
    St<double> s;
    gather(vc, vc, r, k + 1, k + 2, k, s);
    MG5_AT(fc, t) = -cell_residual(s, -MG5_AT(fc, t), cf);   // op + fc
}

// fine interior += trilinear interpolation of (vc - v0c), ghosts included (the
// ghost correction is the extrapolated boundary value kept by the refresh).
// MASKED: cells with mask 0 keep their values.
template <bool MASKED>
__global__ void k_pbox_prolong(const double *__restrict__ vc, const double *__restrict__ v0c, int q0,
                               int q1, int q2, double *__restrict__ vf,
                               const unsigned char *__restrict__ mask)
{
    const int p0 = 2 * q0, p1 = 2 * q1, p2 = 2 * q2;
    const long long total = (long long)p0 * p1 * p2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total || (MASKED && !MG5_AT(mask, t)))
        return;
    const int k = (int)(t % p2);
    const long long q = t / p2;
    const int j = (int)(q % p1), i = (int)(q / p1);
    // coarse box indices of the parent (+1 for the ghost offset) and of its neighbour
    const int P[3] = {(i >> 1) + 1, (j >> 1) + 1, (k >> 1) + 1};
    const int Q[3] = {(i & 1) ? P[0] + 1 : P[0] - 1, (j & 1) ? P[1] + 1 : P[1] - 1,
                      (k & 1) ? P[2] + 1 : P[2] - 1};
    const int d1 = q1 + 2, d2 = q2 + 2;
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const long long idx = bidx(a ? Q[0] : P[0], b ? Q[1] : P[1], c ? Q[2] : P[2], d1, d2);
                const double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (c ? 0.25 : 0.75);
                acc += w * (MG5_AT(vc, idx) - MG5_AT(v0c, idx));
            }
    MG5_AT(vf, bidx(i + 1, j + 1, k + 1, p1 + 2, p2 + 2)) += acc;
}

// coarse box ghost cells: mean of the fine ghost cells each one covers
// (per axis: coarse -1 -> fine -1; coarse q -> fine p; otherwise its two children)
__global__ void k_pbox_ghosts(const double *__restrict__ fb, int p0, int p1, int p2,
                              double *__restrict__ g1, double *__restrict__ g2,
                              double *__restrict__ g3)
{
    const int q[3] = {p0 >> 1, p1 >> 1, p2 >> 1};
    const int D0 = q[0] + 2, D1 = q[1] + 2, D2 = q[2] + 2;
    const long long total = (long long)D0 * D1 * D2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int K = (int)(t % D2);
    const long long qq = t / D2;
    const int J = (int)(qq % D1), I = (int)(qq / D1);
    const int loc[3] = {I - 1, J - 1, K - 1};  // coarse interior index, -1 .. q
    bool ghost = false;
    int lo[3], cnt[3];
    for (int a = 0; a < 3; ++a) {
        if (loc[a] < 0) {
            ghost = true;
            lo[a] = -1;
            cnt[a] = 1;
        } else if (loc[a] >= q[a]) {
            ghost = true;
            lo[a] = 2 * q[a];
            cnt[a] = 1;
        } else {
            lo[a] = 2 * loc[a];
            cnt[a] = 2;
        }
    }
    if (!ghost)
        return;
    double s = 0.0;
    for (int a = 0; a < cnt[0]; ++a)
        for (int b = 0; b < cnt[1]; ++b)
            for (int c = 0; c < cnt[2]; ++c)
                s += MG5_AT(fb, bidx(lo[0] + a + 1, lo[1] + b + 1, lo[2] + c + 1, p1 + 2, p2 + 2));
    const double g = s / (double)(cnt[0] * cnt[1] * cnt[2]);
    MG5_AT(g1, t) = g;
    MG5_AT(g2, t) = g;
    MG5_AT(g3, t) = g;
}

// ghost refresh of a coarse box: v(g) = v0(g) + w^m (v(a) - v0(a))
__device__ __forceinline__ void ghost_refresh_cell(double *v, const double *v0, int I, int J, int K,
                                                   int q0, int q1, int q2, double w)
{
    const int d1 = q1 + 2, d2 = q2 + 2;
    int m = 0;
    int a0 = I, a1 = J, a2 = K;
    if (I == 0) { a0 = 1; ++m; } else if (I == q0 + 1) { a0 = q0; ++m; }
    if (J == 0) { a1 = 1; ++m; } else if (J == q1 + 1) { a1 = q1; ++m; }
    if (K == 0) { a2 = 1; ++m; } else if (K == q2 + 1) { a2 = q2; ++m; }
    if (m == 0)
        return;
    const double wm = m == 1 ? w : (m == 2 ? w * w : w * w * w);
    const long long g = bidx(I, J, K, d1, d2), a = bidx(a0, a1, a2, d1, d2);
    MG5_AT(v, g) = MG5_AT(v0, g) + wm * (MG5_AT(v, a) - MG5_AT(v0, a));
}

// Coarsest patch grid, one CTA: before each sweep the residual norm; stop at
// rtol times the first one or after nu_max sweeps.  A -> B (red) -> A (black).
// Boxes up to kPboxSmemCells cells run in shared memory.  MASKED: cells with mask 0
// are neither relaxed nor counted in the residual norm.
constexpr int kPboxSmemCells = 1024;
constexpr int kPboxThreads = 512;   // 128 registers a thread: stencil offsets stay in registers

template <bool MASKED>
__global__ void __launch_bounds__(kPboxThreads)
    k_pbox_coarsest(double *A, double *B, const double *__restrict__ f, int p0, int p1, int p2,
                    CoefT<double> cf, int nu_max, double rtol, unsigned long long *clamp,
                    int *sweeps_out, const double *__restrict__ v0, double w,
                    const unsigned char *__restrict__ mask)
{
    extern __shared__ __align__(16) unsigned char pb_raw[];
    __shared__ double bc_s;
    const int n3 = p0 * p1 * p2;
    const int d1 = p1 + 2, d2 = p2 + 2;
    const int nbox = (p0 + 2) * d1 * d2;
    const bool in_smem = nbox <= kPboxSmemCells;
    double *a = A, *b = B;
    const double *ff = f, *g0 = v0;
    if (in_smem) {
        double *sm = reinterpret_cast<double *>(pb_raw);
        a = sm;
        b = sm + nbox;
        double *sf = sm + 2 * nbox;
        double *sv0 = sm + 3 * nbox;
        for (int q = threadIdx.x; q < nbox; q += blockDim.x) {
            MG5_AT(a, q) = MG5_AT(A, q);
            MG5_AT(b, q) = MG5_AT(B, q);
            if (v0)
                MG5_AT(sv0, q) = MG5_AT(v0, q);
            if (q < n3)
                MG5_AT(sf, q) = MG5_AT(f, q);
        }
        ff = sf;
        g0 = v0 ? sv0 : nullptr;
        __syncthreads();
    }
    // coarse grids keep their ghosts on the extrapolated boundary condition
    auto refresh = [&](double *X) {
        if (!g0)
            return;
        for (int g = threadIdx.x; g < nbox; g += blockDim.x) {
            const int K = g % d2, J = (g / d2) % d1, I = g / (d1 * d2);
            ghost_refresh_cell(X, g0, I, J, K, p0, p1, p2, w);
        }
        __syncthreads();
    };
    refresh(a);
    double r0 = -1.0;
    int it = 0;
    unsigned long long my_clamps = 0;
    constexpr int kOwnGhosts = 8;
    if (in_smem && n3 <= (int)blockDim.x && nbox <= kOwnGhosts * (int)blockDim.x) {
        // one interior cell per thread and at most kOwnGhosts box cells: stencil offsets,
        // colour, f and the ghost-refresh terms once (the same values as the loop below)
        const int p = threadIdx.x;
        const bool mine = p < n3;
        const bool active = mine && (!MASKED || MG5_AT(mask, p));
        Nbr nb{};
        int colour_me = 0, cbox = 0;
        double fme = 0.0;
        if (mine) {
            const int k = p % p2, j = (p / p2) % p1, i = p / (p1 * p2);
            nb = nbr_of(box_rows(d1, d2, i + 1, j + 1), k + 1, k + 2, k);
            colour_me = (i + j + k) & 1;
            cbox = nb.o[0];
            fme = MG5_AT(ff, p);
        }
        // slot e covers box cell threadIdx.x + e * blockDim.x; gi < 0: not a ghost (or none)
        int gi[kOwnGhosts], ga[kOwnGhosts];
        double gw[kOwnGhosts];
#pragma unroll
        for (int e = 0; e < kOwnGhosts; ++e) {
            gi[e] = -1;
            ga[e] = 0;
            gw[e] = 0.0;
            const int q = threadIdx.x + e * blockDim.x;
            if (!g0 || q >= nbox)
                continue;
            const int K = q % d2, J = (q / d2) % d1, I = q / (d1 * d2);
            int m = 0, a0 = I, a1 = J, a2 = K;
            if (I == 0) { a0 = 1; ++m; } else if (I == p0 + 1) { a0 = p0; ++m; }
            if (J == 0) { a1 = 1; ++m; } else if (J == p1 + 1) { a1 = p1; ++m; }
            if (K == 0) { a2 = 1; ++m; } else if (K == p2 + 1) { a2 = p2; ++m; }
            if (m == 0)
                continue;
            gi[e] = q;
            ga[e] = (a0 * d1 + a1) * d2 + a2;
            gw[e] = m == 1 ? w : (m == 2 ? w * w : w * w * w);
        }
        auto refresh_own = [&](double *X) {
#pragma unroll
            for (int e = 0; e < kOwnGhosts; ++e)
                if (gi[e] >= 0)
                    MG5_AT(X, gi[e]) = MG5_AT(g0, gi[e]) + gw[e] * (MG5_AT(X, ga[e]) - MG5_AT(g0, ga[e]));
            __syncthreads();
        };
        for (; it < nu_max; ++it) {
            double2 acc = make_double2(0.0, 0.0);
            if (active) {
                St<double> s;
                gather_nbr((const double *)a, nb, s);
                const double res = cell_residual(s, fme, cf);
                acc.y = res * res;
            }
            acc = block_sum2(acc);
            if (threadIdx.x == 0)
                bc_s = acc.y;
            __syncthreads();
            const double rn = sqrt(bc_s);
            __syncthreads();
            if (r0 < 0.0)
                r0 = rn;
            if (rn <= rtol * r0)
                break;
            for (int colour = 0; colour < 2; ++colour) {
                const double *src = colour == 0 ? a : b;
                double *dst = colour == 0 ? b : a;
                if (mine) {
                    if (colour_me != colour || !active) {
                        MG5_AT(dst, cbox) = MG5_AT(src, cbox);
                    } else {
                        St<double> s;
                        gather_nbr(src, nb, s);
                        bool cl = false;
                        MG5_AT(dst, cbox) = cell_update(s, fme, cf, cl);
                        my_clamps += cl ? 1ull : 0ull;
                    }
                }
                __syncthreads();
                if (g0)
                    refresh_own(dst);
            }
        }
        nu_max = 0;   // skip the general loop
    }
    for (; it < nu_max; ++it) {
        double2 acc = make_double2(0.0, 0.0);
        for (int p = threadIdx.x; p < n3; p += blockDim.x) {
            if (MASKED && !MG5_AT(mask, p))
                continue;
            const int k = p % p2, j = (p / p2) % p1, i = p / (p1 * p2);
            const Rows r = box_rows(d1, d2, i + 1, j + 1);
            St<double> s;
            gather((const double *)a, (const double *)a, r, k + 1, k + 2, k, s);
            const double res = cell_residual(s, MG5_AT(ff, p), cf);
            acc.y += res * res;
        }
        acc = block_sum2(acc);
        if (threadIdx.x == 0)
            bc_s = acc.y;
        __syncthreads();
        const double rn = sqrt(bc_s);
        __syncthreads();
        if (r0 < 0.0)
            r0 = rn;
        if (rn <= rtol * r0)
            break;
        for (int colour = 0; colour < 2; ++colour) {
            const double *src = colour == 0 ? a : b;
            double *dst = colour == 0 ? b : a;
            for (int p = threadIdx.x; p < n3; p += blockDim.x) {
                const int k = p % p2, j = (p / p2) % p1, i = p / (p1 * p2);
                const Rows r = box_rows(d1, d2, i + 1, j + 1);
                if (((i + j + k) & 1) != colour || (MASKED && !MG5_AT(mask, p))) {
                    MG5_AT(dst, r.r00 + k + 1) = MG5_AT(src, r.r00 + k + 1);
                    continue;
                }
                St<double> s;
                gather(src, src, r, k + 1, k + 2, k, s);
                bool cl = false;
                MG5_AT(dst, r.r00 + k + 1) = cell_update(s, MG5_AT(ff, p), cf, cl);
                my_clamps += cl ? 1ull : 0ull;
            }
            __syncthreads();
            refresh(dst);
        }
    }
    if (in_smem) {
        for (int q = threadIdx.x; q < nbox; q += blockDim.x)
            MG5_AT(A, q) = MG5_AT(a, q);
    }
    if (my_clamps)
        atomicAdd(&MG5_AT(clamp, 0), my_clamps);
    if (threadIdx.x == 0 && sweeps_out)
        atomicAdd(&MG5_AT(sweeps_out, 0), it);
}

// ---------------------------------------------------------------- launchers

cudaError_t launch_pbox_resid_restrict(const double *v, const double *f, const int p[3],
                                       CoefT<double> cf, double *vc, double *v0c, double *fc,
                                       double2 *partials, int *nblocks, cudaStream_t st,
                                       const unsigned char *mask, const Fin &fin)
{
    const long long work = (long long)(p[0] / 2) * (p[1] / 2) * (p[2] / 2);
    int g;
    if (8 * work <= kChildMaxFine) {   // a thread per fine cell
        const int bs = block_spread(8 * work);
        g = grid_spread(8 * work);
        if (g > kReduceBlocksFp64)
            g = kReduceBlocksFp64;
        if (mask)
            k_pbox_resid_restrict_child<true><<<g, bs, 0, st>>>(v, f, p[0], p[1], p[2], cf, vc,
                                                                v0c, fc, partials, mask, fin);
        else
            k_pbox_resid_restrict_child<false><<<g, bs, 0, st>>>(v, f, p[0], p[1], p[2], cf, vc,
                                                                 v0c, fc, partials, mask, fin);
    } else {   // a thread per coarse cell, blocks of kBlock (fewer partials to combine)
        g = blocks_for(work);
        if (g > kReduceBlocksFp64)
            g = kReduceBlocksFp64;
        if (mask)
            k_pbox_resid_restrict<true><<<g, kBlock, 0, st>>>(v, f, p[0], p[1], p[2], cf, vc, v0c,
                                                              fc, partials, mask, fin);
        else
            k_pbox_resid_restrict<false><<<g, kBlock, 0, st>>>(v, f, p[0], p[1], p[2], cf, vc, v0c,
                                                               fc, partials, mask, fin);
    }
    *nblocks = g;
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pbox_coarse_rhs(const double *vc, double *fc, const int q[3], CoefT<double> cf,
                                   cudaStream_t st)
{
    const long long work = (long long)q[0] * q[1] * q[2];
    k_pbox_coarse_rhs<<<grid_spread(work), block_spread(work), 0, st>>>(vc, fc, q[0], q[1], q[2], cf);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pbox_prolong(const double *vc, const double *v0c, const int q[3], double *vf,
                                cudaStream_t st, const unsigned char *mask)
{
    const long long work = 8ll * q[0] * q[1] * q[2];
    if (mask)
        k_pbox_prolong<true><<<grid_spread(work), block_spread(work), 0, st>>>(vc, v0c, q[0], q[1], q[2], vf,
                                                                  mask);
    else
        k_pbox_prolong<false><<<grid_spread(work), block_spread(work), 0, st>>>(vc, v0c, q[0], q[1], q[2], vf,
                                                                   mask);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pbox_ghosts(const double *fine_box, const int p[3], double *g1, double *g2,
                               double *g3, cudaStream_t st)
{
    const long long work = (long long)(p[0] / 2 + 2) * (p[1] / 2 + 2) * (p[2] / 2 + 2);
    k_pbox_ghosts<<<grid_spread(work), block_spread(work), 0, st>>>(fine_box, p[0], p[1], p[2], g1, g2, g3);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_pbox_coarsest(double *A, double *B, const double *f, const int p[3],
                                 CoefT<double> cf, int nu_max, double rtol, unsigned long long *clamp,
                                 int *sweeps, cudaStream_t st, const double *v0, double w,
                                 const unsigned char *mask)
{
    const int n3 = p[0] * p[1] * p[2];
    const int nbox = (p[0] + 2) * (p[1] + 2) * (p[2] + 2);
    int threads = ((n3 + 31) / 32) * 32;
    if (threads > kPboxThreads)
        threads = kPboxThreads;
    const size_t sm = nbox <= kPboxSmemCells ? (size_t)4 * nbox * sizeof(double) : 0;
    if (mask)
        k_pbox_coarsest<true><<<1, threads, sm, st>>>(A, B, f, p[0], p[1], p[2], cf, nu_max, rtol,
                                                      clamp, sweeps, v0, w, mask);
    else
        k_pbox_coarsest<false><<<1, threads, sm, st>>>(A, B, f, p[0], p[1], p[2], cf, nu_max, rtol,
                                                       clamp, sweeps, v0, w, mask);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace mg5
