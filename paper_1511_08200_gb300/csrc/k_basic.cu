// k_basic.cu -- the plain (one thread per cell) kernels of the mg5 hot path:
// snapshot red-black sweep, operator, residual (+ fused 8-child restriction),
// FAS coarse right-hand side, trilinear prolongation + correction, the
// single-CTA coarsest-grid solve, reductions, force, coarse->fine
// interpolation and the Dirichlet patch sweep.
//
// Paper: arXiv:1511.08200, Eq. (eomvarphi), Eq. (newton), Sec. 3.1 (level
// solve, V-cycles, boundary values from the coarser level), Sec. 3.2
// (interpolated fine phi, force by central differences).
#include "mg5_fin.cuh"

namespace mg5 {


// --------------------------------------------------------------------------
// snapshot red-black sweep: two passes.
// Red pass: red cells ((i+j+k) even) from `in` into `out`.
// Black pass: faces (red, new) from `out`, the centre and the edges (black, old) from `in`,
// into `out`; between them the two passes write every cell of `out` once.
// Each thread owns the pair (2kk, 2kk+1) of one row, one cell of each colour.
// --------------------------------------------------------------------------
template <typename T, bool BASE>
__global__ void k_sweep_red(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ f,
                            const double *__restrict__ cptr, int n, CoefT<T> cf,
                            unsigned long long *clamp, const T *__restrict__ B)
{
    const int half = n >> 1;
    const long long total = (long long)n * n * half;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int kk = (int)(t % half);
    const long long q = t / half;
    const int j = (int)(q % n), i = (int)(q / n);
    const int par = (i + j) & 1;
    const int kr = 2 * kk + par;
    const Rows r = periodic_rows(n, i, j);
    const int kp = (kr == n - 1) ? 0 : kr + 1, km = (kr == 0) ? n - 1 : kr - 1;
    St<T> s, sb;
    gather(in, in, r, kr, kp, km, s);
    if constexpr (BASE)
        gather(B, B, r, kr, kp, km, sb);
    bool cl = false;
    const T v = upd<T, BASE>(s, sb, MG5_AT(f, r.r00 + kr) + (T)(MG5_AT(cptr, 0)), cf, cl);
    MG5_AT(out, r.r00 + kr) = v;
    if (cl)
        atomicAdd(&MG5_AT(clamp, 0), 1ull);
}

template <typename T, bool BASE>
__global__ void k_sweep_black(const T *__restrict__ in, T *out, const T *__restrict__ f,
                              const double *__restrict__ cptr, int n, CoefT<T> cf,
                              unsigned long long *clamp, const T *__restrict__ B)
{
    const int half = n >> 1;
    const long long total = (long long)n * n * half;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int kk = (int)(t % half);
    const long long q = t / half;
    const int j = (int)(q % n), i = (int)(q / n);
    const int kb = 2 * kk + 1 - ((i + j) & 1);
    const Rows r = periodic_rows(n, i, j);
    const int kp = (kb == n - 1) ? 0 : kb + 1, km = (kb == 0) ? n - 1 : kb - 1;
    St<T> s, sb;
    gather3((const T *)out, in, in, r, kb, kp, km, s);
    if constexpr (BASE)
        gather(B, B, r, kb, kp, km, sb);
    bool cl = false;
    const T v = upd<T, BASE>(s, sb, MG5_AT(f, r.r00 + kb) + (T)(MG5_AT(cptr, 0)), cf, cl);
    MG5_AT(out, r.r00 + kb) = v;
    if (cl)
        atomicAdd(&MG5_AT(clamp, 0), 1ull);
}

template <typename T>
cudaError_t launch_sweep(const T *in, T *out, const T *f, const double *cptr, int n, CoefT<T> cf,
                         unsigned long long *clamp, cudaStream_t st, const T *B, int block)
{
    if (block < 32 || block > 1024 || block % 32)
        return cudaErrorInvalidValue;
    const long long work = (long long)n * n * (n / 2);
    const int g = (int)((work + block - 1) / block);
    if (B) {
        k_sweep_red<T, true><<<g, block, 0, st>>>(in, out, f, cptr, n, cf, clamp, B);
        k_sweep_black<T, true><<<g, block, 0, st>>>(in, out, f, cptr, n, cf, clamp, B);
    } else {
        k_sweep_red<T, false><<<g, block, 0, st>>>(in, out, f, cptr, n, cf, clamp, B);
        k_sweep_black<T, false><<<g, block, 0, st>>>(in, out, f, cptr, n, cf, clamp, B);
    }
    count_launch(2);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// operator and residual
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_operator(const T *__restrict__ phi, int n, CoefT<T> cf, T *__restrict__ out)
{
    const long long total = (long long)n * n * n;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int k = (int)(t % n);
    const long long q = t / n;
    const int j = (int)(q % n), i = (int)(q / n);
    const Rows r = periodic_rows(n, i, j);
    const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
    St<T> s;
    gather(phi, phi, r, k, kp, km, s);
    MG5_AT(out, t) = cell_op(s, cf);
}

template <typename T>
cudaError_t launch_operator(const T *phi, int n, CoefT<T> cf, T *out, cudaStream_t st)
{
    const long long work = (long long)n * n * n;
    k_operator<T><<<grid_spread(work), block_spread(work), 0, st>>>(phi, n, cf, out);
    count_launch(1);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_residual(const T *__restrict__ phi, const T *__restrict__ f,
                           const double *__restrict__ cptr, int n, CoefT<T> cf, T *__restrict__ r_out,
                           Moments *__restrict__ partials, Fin fin)
{
    const long long total = (long long)n * n * n;
    const double c = MG5_AT(cptr, 0);
    MomAcc<T> acc;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t % n);
        const long long q = t / n;
        const int j = (int)(q % n), i = (int)(q / n);
        const Rows r = periodic_rows(n, i, j);
        const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
        St<T> s;
        gather(phi, phi, r, k, kp, km, s);
        const T res = cell_residual(s, MG5_AT(f, t) + (T)c, cf);
        if (r_out)
            MG5_AT(r_out, t) = res;
        acc.add(res);
    }
    const Moments m = block_moments(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = m;
    if (fin.ls)
        finalize_if_last(reinterpret_cast<double2 *>(partials), fin);
}

template <typename T>
cudaError_t launch_residual(const T *phi, const T *f, const double *cptr, int n, CoefT<T> cf, T *r,
                            double2 *partials, int *nblocks, cudaStream_t st, const Fin &fin)
{
    const long long work = (long long)n * n * n;
    const int cap = sizeof(T) == 8 ? kReduceBlocksFp64 : kReduceBlocks;
    const int bs = block_spread(work);
    int g = grid_spread(work);
    if (g > cap)
        g = cap;
    k_residual<T><<<g, bs, 0, st>>>(phi, f, cptr, n, cf, r, reinterpret_cast<Moments *>(partials),
                                        fin);
    *nblocks = g;
    count_launch(1);
    return cudaGetLastError();
}

// Residual of the 8 children of each coarse cell, restricted with v.
template <typename T, bool BASE>
__global__ void k_resid_restrict(const T *__restrict__ v, const T *__restrict__ f,
                                 const double *__restrict__ cptr, int n, CoefT<T> cf,
                                 T *__restrict__ vc, T *__restrict__ v0c, T *__restrict__ rc,
                                 Moments *__restrict__ partials, const T *__restrict__ B, Fin fin)
{
    const int nc = n >> 1;
    const long long total = (long long)nc * nc * nc;
    const double c = MG5_AT(cptr, 0);
    MomAcc<T> acc;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int K = (int)(t % nc);
        const long long q = t / nc;
        const int J = (int)(q % nc), I = (int)(q / nc);
        T sv = 0, sr = 0;
#pragma unroll 2
        for (int ch = 0; ch < 8; ++ch) {
            const int i = 2 * I + (ch >> 2), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch & 1);
            const Rows r = periodic_rows(n, i, j);
            const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
            St<T> s, sb;
            gather(v, v, r, k, kp, km, s);
            if constexpr (BASE)
                gather(B, B, r, k, kp, km, sb);
            const T res = resid_of<T, BASE>(s, sb, MG5_AT(f, r.r00 + k) + (T)c, cf);
            sv += s.c;
            sr += res;
            acc.add(res);
        }
        const T mv = sv * (T)0.125;
        MG5_AT(vc, t) = mv;
        MG5_AT(v0c, t) = mv;
        MG5_AT(rc, t) = sr * (T)0.125;
    }
    const Moments m = block_moments(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = m;
    if (fin.ls)
        finalize_if_last(reinterpret_cast<double2 *>(partials), fin);
}

// The same residual and restriction with a thread per fine cell, for the coarse grids of the
// FP64 solves (up to kChildMaxFine fine cells; above that the FP64 pipe, not the chain, sets
// the time, and the butterfly's extra adds made the 64^3 and 128^3 launches slower): eight
// consecutive lanes hold the eight children of one coarse cell (child ch = lane & 7, its i, j
// and k offsets ch >> 2, (ch >> 1) & 1 and ch & 1) and sum their centres and residuals by
// three butterfly shuffles, ((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7)).  A thread
// computes one FP64 residual instead of a chain of eight: GB300 runs FP64 at 2 lanes a clock
// per SM, and on the coarse grids, whose blocks reach few SMs, that chain set the time.  The
// loop runs over whole warps (four coarse cells a warp a pass), so every lane reaches the
// shuffles.
__global__ void k_resid_restrict_child(const double *__restrict__ v, const double *__restrict__ f,
                                       const double *__restrict__ cptr, int n, CoefT<double> cf,
                                       double *__restrict__ vc, double *__restrict__ v0c,
                                       double *__restrict__ rc, Moments *__restrict__ partials,
                                       Fin fin)
{
    const int nc = n >> 1;
    const long long total = (long long)nc * nc * nc;
    const double c = MG5_AT(cptr, 0);
    const int lane = threadIdx.x & 31, ch = lane & 7;
    const long long stride = (long long)gridDim.x * blockDim.x / 8;   // coarse cells a pass
    MomAcc<double> acc;
    for (long long t0 = ((long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) / 8; t0 < total;
         t0 += stride) {
        const long long t = t0 + (lane >> 3);
        const bool live = t < total;
        double cv = 0.0, res = 0.0;
        if (live) {
            const int K = (int)(t % nc);
            const long long q = t / nc;
            const int J = (int)(q % nc), I = (int)(q / nc);
            const int i = 2 * I + (ch >> 2), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch & 1);
            const Rows r = periodic_rows(n, i, j);
            const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
            St<double> s;
            gather(v, v, r, k, kp, km, s);
            res = resid_of<double, false>(s, s, MG5_AT(f, r.r00 + k) + c, cf);
            cv = s.c;
            acc.add(res);
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            cv += __shfl_xor_sync(0xffffffffu, cv, o);
            res += __shfl_xor_sync(0xffffffffu, res, o);
        }
        if (live && ch == 0) {
            const double mv = cv * 0.125;
            MG5_AT(vc, t) = mv;
            MG5_AT(v0c, t) = mv;
            MG5_AT(rc, t) = res * 0.125;
        }
    }
    const Moments m = block_moments(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = m;
    if (fin.ls)
        finalize_if_last(reinterpret_cast<double2 *>(partials), fin);
}

template <typename T>
cudaError_t launch_resid_restrict(const T *v, const T *f, const double *cptr, int n, CoefT<T> cf,
                                  T *vc, T *v0c, T *rc, double2 *partials, int *nblocks,
                                  cudaStream_t st, const T *B, const Fin &fin)
{
    const long long work = (long long)(n / 2) * (n / 2) * (n / 2);
    const int cap = sizeof(T) == 8 ? kReduceBlocksFp64 : kReduceBlocks;
    if constexpr (sizeof(T) == 8) {
        if (!B && 8 * work <= kChildMaxFine) {   // coarse grids of the FP64 solves
            const long long fine = 8 * work;
            const int bf = block_spread(fine);
            int gf = grid_spread(fine);
            if (gf > cap)
                gf = cap;
            k_resid_restrict_child<<<gf, bf, 0, st>>>(v, f, cptr, n, cf, vc, v0c, rc,
                                                      reinterpret_cast<Moments *>(partials), fin);
            *nblocks = gf;
            count_launch(1);
            return cudaGetLastError();
        }
    }
    // blocks of kBlock: spreading the coarse cells over more, smaller blocks measured slower
    // here (more partials for the last block to combine)
    int g = blocks_for(work);
    if (g > cap)
        g = cap;
    const int bs = kBlock;
    Moments *mp = reinterpret_cast<Moments *>(partials);
    if (B)
        k_resid_restrict<T, true><<<g, bs, 0, st>>>(v, f, cptr, n, cf, vc, v0c, rc, mp, B, fin);
    else
        k_resid_restrict<T, false><<<g, bs, 0, st>>>(v, f, cptr, n, cf, vc, v0c, rc, mp, B, fin);
    *nblocks = g;
    count_launch(1);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_restrict(const T *__restrict__ fine, int n, T *__restrict__ coarse)
{
    const int nc = n >> 1;
    const long long total = (long long)nc * nc * nc;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int K = (int)(t % nc);
    const long long q = t / nc;
    const int J = (int)(q % nc), I = (int)(q / nc);
    T s = 0;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        const long long i = 2 * I + (ch >> 2), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch & 1);
        s += MG5_AT(fine, (i * n + j) * n + k);
    }
    MG5_AT(coarse, t) = s * (T)0.125;
}

template <typename T>
cudaError_t launch_restrict(const T *fine, int n, T *coarse, cudaStream_t st)
{
    const long long work = (long long)(n / 2) * (n / 2) * (n / 2);
    k_restrict<T><<<grid_spread(work), block_spread(work), 0, st>>>(fine, n, coarse);
    count_launch(1);
    return cudaGetLastError();
}

// fc = op_c(vc) + fc - m ; the coarse c restarts at zero.
template <typename T, bool BASE>
__global__ void k_coarse_rhs(const T *__restrict__ vc, T *__restrict__ fc,
                             const double *__restrict__ m_fine, double *__restrict__ c_coarse,
                             int nc, CoefT<T> cf, const T *__restrict__ B)
{
    const long long total = (long long)nc * nc * nc;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0)
        MG5_AT(c_coarse, 0) = 0.0;
    if (t >= total)
        return;
    const int k = (int)(t % nc);
    const long long q = t / nc;
    const int j = (int)(q % nc), i = (int)(q / nc);
    const Rows r = periodic_rows(nc, i, j);
    const int kp = (k == nc - 1) ? 0 : k + 1, km = (k == 0) ? nc - 1 : k - 1;
    St<T> s, sb;
    gather(vc, vc, r, k, kp, km, s);
    if constexpr (BASE)
        gather(B, B, r, k, kp, km, sb);
    if constexpr (BASE)
        MG5_AT(fc, t) = opr<T, BASE>(s, sb, cf) + MG5_AT(fc, t) - (T)(MG5_AT(m_fine, 0));
    else   // op + fc - m as -(m - fc - op): the residual chain's FP64 operation count
        MG5_AT(fc, t) = -cell_residual(s, (T)(MG5_AT(m_fine, 0)) - MG5_AT(fc, t), cf);
}

template <typename T>
cudaError_t launch_coarse_rhs(const T *vc, T *fc, const double *m_fine, double *c_coarse, int nc,
                              CoefT<T> cfc, cudaStream_t st, const T *B)
{
    const long long work = (long long)nc * nc * nc;
    if (B)
        k_coarse_rhs<T, true><<<grid_spread(work), block_spread(work), 0, st>>>(vc, fc, m_fine, c_coarse, nc, cfc, B);
    else
        k_coarse_rhs<T, false><<<grid_spread(work), block_spread(work), 0, st>>>(vc, fc, m_fine, c_coarse, nc, cfc, B);
    count_launch(1);
    return cudaGetLastError();
}

// Cell-centred trilinear prolongation: along each axis a fine centre is a
// quarter coarse cell from its parent, so it takes 3/4 of the parent and 1/4
// of the parent's neighbour on its own side.  One thread per coarse cell reads
// the 3x3x3 coarse neighbourhood once and writes its 8 children, applying the
// separable weights along k, then j, then i; the two children along k are one
// vector read-modify-write.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename T>
__global__ void k_prolong_add(const T *__restrict__ vc, const T *__restrict__ v0c, int nc,
                              T *__restrict__ vf, double *c_fine, const double *c_coarse)
{
    const long long total = (long long)nc * nc * nc;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && c_fine && c_coarse)
        MG5_AT(c_fine, 0) += MG5_AT(c_coarse, 0);
    if (t >= total)
        return;
    const int K = (int)(t % nc);
    const long long q = t / nc;
    const int J = (int)(q % nc), I = (int)(q / nc);
    const long long NC = nc;
    int ii[3], jj[3], kk[3];
    ii[0] = I == 0 ? nc - 1 : I - 1, ii[1] = I, ii[2] = I == nc - 1 ? 0 : I + 1;
    jj[0] = J == 0 ? nc - 1 : J - 1, jj[1] = J, jj[2] = J == nc - 1 ? 0 : J + 1;
    kk[0] = K == 0 ? nc - 1 : K - 1, kk[1] = K, kk[2] = K == nc - 1 ? 0 : K + 1;
    // Weights (3/4, 1/4) per axis, applied as 3 x + y with the three factors 1/4 folded into
    // one 1/64 at the end: one FP64 multiply-add a stage instead of a multiply and an add
    // (the FP64 correction is FP64-pipe bound on GB300).  Along k: Z[a][b][c] for child c
    // (0: 2K, 1: 2K+1).
    T Z[3][3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const long long row = ((long long)ii[a] * NC + jj[b]) * NC;
            T e[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                e[c] = v0c ? MG5_AT(vc, row + kk[c]) - MG5_AT(v0c, row + kk[c]) : MG5_AT(vc, row + kk[c]);
            Z[a][b][0] = fma((T)3, e[1], e[0]);
            Z[a][b][1] = fma((T)3, e[1], e[2]);
        }
    // along j: Y[a][cj][ck], shared by both children along i
    T Y[3][2][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int cj = 0; cj < 2; ++cj)
#pragma unroll
            for (int ck = 0; ck < 2; ++ck)
                Y[a][cj][ck] = fma((T)3, Z[a][1][ck], Z[a][cj ? 2 : 0][ck]);
    const int n = 2 * nc;
    const T w = (T)(1.0 / 64.0);
#pragma unroll
    for (int ci = 0; ci < 2; ++ci)
#pragma unroll
        for (int cj = 0; cj < 2; ++cj) {
            T out[2];
#pragma unroll
            for (int ck = 0; ck < 2; ++ck)
                out[ck] = fma((T)3, Y[1][cj][ck], Y[ci ? 2 : 0][cj][ck]);
            const long long f = ((long long)(2 * I + ci) * n + (2 * J + cj)) * n + 2 * K;
            using V = typename Vec2<T>::type;
            V *p = &MG5_AT(reinterpret_cast<V *>(vf + f), 0);
            V v = *p;
            v.x = fma(out[0], w, v.x);
            v.y = fma(out[1], w, v.y);
            *p = v;
        }
}

// The same prolongation as a march along i (coarse sides >= 128): one thread per coarse
// column (J, K) over a chunk of coarse planes.  The k- and j-stages of a coarse plane (Y[cj][ck] below, the values of
// k_prolong_add's Y for that plane) are formed once when the plane enters and kept for the
// three coarse planes that use them, so each coarse value is read and differenced once per
// chunk instead of 27 times and each stage runs once per plane; the i-stage and the fine
// update are k_prolong_add's, so both kernels give the same values.
template <typename T>
__global__ void k_prolong_march(const T *__restrict__ vc, const T *__restrict__ v0c, int nc,
                                int ichunk, T *__restrict__ vf, double *c_fine,
                                const double *c_coarse)
{
    const int K = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = blockIdx.y;
    const int I0 = blockIdx.z * ichunk;
    const int I1 = min(I0 + ichunk, nc);
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && c_fine &&
        c_coarse)
        MG5_AT(c_fine, 0) += MG5_AT(c_coarse, 0);
    if (K >= nc)
        return;
    const long long NC = nc;
    const int kk[3] = {K == 0 ? nc - 1 : K - 1, K, K == nc - 1 ? 0 : K + 1};
    const int jj[3] = {J == 0 ? nc - 1 : J - 1, J, J == nc - 1 ? 0 : J + 1};
    // Y[cj][ck] of coarse plane i
    auto yplane = [&](int i, T y[2][2]) {
        T Z[3][2];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const long long row = ((long long)i * NC + jj[b]) * NC;
            T e[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                e[c] = v0c ? MG5_AT(vc, row + kk[c]) - MG5_AT(v0c, row + kk[c]) : MG5_AT(vc, row + kk[c]);
            Z[b][0] = fma((T)3, e[1], e[0]);
            Z[b][1] = fma((T)3, e[1], e[2]);
        }
#pragma unroll
        for (int cj = 0; cj < 2; ++cj)
#pragma unroll
            for (int ck = 0; ck < 2; ++ck)
                y[cj][ck] = fma((T)3, Z[1][ck], Z[cj ? 2 : 0][ck]);
    };
    T ym[2][2], y0[2][2], yp[2][2];   // planes I - 1, I, I + 1
    yplane(I0 == 0 ? nc - 1 : I0 - 1, ym);
    yplane(I0, y0);
    const int n = 2 * nc;
    const T w = (T)(1.0 / 64.0);
    using V = typename Vec2<T>::type;
    for (int I = I0; I < I1; ++I) {
        yplane(I == nc - 1 ? 0 : I + 1, yp);
#pragma unroll
        for (int ci = 0; ci < 2; ++ci)
#pragma unroll
            for (int cj = 0; cj < 2; ++cj) {
                const T o0 = fma((T)3, y0[cj][0], ci ? yp[cj][0] : ym[cj][0]);
                const T o1 = fma((T)3, y0[cj][1], ci ? yp[cj][1] : ym[cj][1]);
                const long long f = ((long long)(2 * I + ci) * n + (2 * J + cj)) * n + 2 * K;
                V *p = &MG5_AT(reinterpret_cast<V *>(vf + f), 0);
                V v = *p;
                v.x = fma(o0, w, v.x);
                v.y = fma(o1, w, v.y);
                *p = v;
            }
#pragma unroll
        for (int cj = 0; cj < 2; ++cj)
#pragma unroll
            for (int ck = 0; ck < 2; ++ck) {
                ym[cj][ck] = y0[cj][ck];
                y0[cj][ck] = yp[cj][ck];
            }
    }
}

template <typename T>
cudaError_t launch_prolong_add(const T *vc, const T *v0c, int nc, T *vf, double *c_fine,
                               const double *c_coarse, cudaStream_t st)
{
    if (nc >= 128) {
        // columns (J, K) x chunks of planes: about a million threads, chunks of >= 4 planes.
        // Below 128^3 coarse cells the gather kernel's four times as many threads hide more
        // latency than the march saves (measured: a 128^3 FP64 solve's prolongations took
        // 0.56 ms with the march, 0.49 ms with the gather; at 512^3 the march halved them)
        const int tx = nc < 256 ? ((nc + 31) / 32) * 32 : 256;
        int chunks = (int)((1ll << 20) / ((long long)nc * nc));
        if (chunks > nc / 4)
            chunks = nc / 4;
        if (chunks < 1)
            chunks = 1;
        const int ichunk = (nc + chunks - 1) / chunks;
        chunks = (nc + ichunk - 1) / ichunk;
        dim3 grid((nc + tx - 1) / tx, nc, chunks);
        k_prolong_march<T><<<grid, tx, 0, st>>>(vc, v0c, nc, ichunk, vf, c_fine, c_coarse);
    } else {
        const long long work = (long long)nc * nc * nc;
        k_prolong_add<T><<<grid_spread(work), block_spread(work), 0, st>>>(vc, v0c, nc, vf, c_fine, c_coarse);
    }
    count_launch(1);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// coarsest grid: one CTA.  Before each sweep: c = mean(op(v) - f) and the
// residual norm; stop when it is <= rtol times the first one or after
// nu_max sweeps.  Sweeps ping-pong A -> B (red) -> A (black) with barriers.
// Grids up to kCoarsestSmemCells cells run entirely in shared memory.
// --------------------------------------------------------------------------
constexpr int kCoarsestThreads = 512;   // 128 registers a thread: stencil offsets stay in registers
constexpr int kCoarsestSmemCells = 1024;   // 4 arrays x 1024 x 8 B = 32 KB

template <typename T, bool BASE>
__global__ void __launch_bounds__(kCoarsestThreads)
    k_coarsest(T *A, T *B, const T *f, int n, CoefT<T> cf, double *cptr, int nu_max, double rtol,
               unsigned long long *clamp, int *sweeps_out, const T *__restrict__ base)
{
    extern __shared__ __align__(16) unsigned char cs_raw[];
    __shared__ double bc_s[2];
    const int n3 = n * n * n;
    const bool in_smem = n3 <= kCoarsestSmemCells;
    T *a = A, *b = B;
    const T *ff = f, *bs = base;
    if (in_smem) {
        T *sm = reinterpret_cast<T *>(cs_raw);
        a = sm;
        b = sm + n3;
        T *sf = sm + 2 * n3;
        T *sbase = sm + 3 * n3;
        for (int p = threadIdx.x; p < n3; p += blockDim.x) {
            MG5_AT(a, p) = MG5_AT(A, p);
            MG5_AT(sf, p) = MG5_AT(f, p);
            if constexpr (BASE)
                MG5_AT(sbase, p) = MG5_AT(base, p);
        }
        ff = sf;
        bs = sbase;
        __syncthreads();
    }
    const double inv_n3 = 1.0 / (double)n3;
    double r0 = -1.0, c = 0.0;
    int it = 0;
    unsigned long long my_clamps = 0;
    if (in_smem && n3 <= (int)blockDim.x) {
        // one cell per thread: its stencil offsets, colour and f once, then only the
        // arithmetic and the barriers per iteration (the same values as the loop below)
        const int p = threadIdx.x;
        const bool mine = p < n3;
        Nbr nb{};
        int colour_me = 0;
        T fme = (T)0;
        if (mine) {
            const int k = p % n, j = (p / n) % n, i = p / (n * n);
            const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
            nb = nbr_of(periodic_rows(n, i, j), k, kp, km);
            colour_me = (i + j + k) & 1;
            fme = MG5_AT(ff, p);
        }
        for (; it < nu_max; ++it) {
            double2 acc = make_double2(0.0, 0.0);
            if (mine) {
                St<T> s, sb;
                gather_nbr((const T *)a, nb, s);
                if constexpr (BASE)
                    gather_nbr(bs, nb, sb);
                const double res = (double)resid_of<T, BASE>(s, sb, fme, cf);
                acc.x = res;
                acc.y = res * res;
            }
            acc = block_sum2(acc);
            if (threadIdx.x == 0) {
                bc_s[0] = acc.x;
                bc_s[1] = acc.y;
            }
            __syncthreads();
            const double m = bc_s[0] * inv_n3;
            const double q2 = bc_s[1] - (double)n3 * m * m;
            const double rn = sqrt(q2 > 0.0 ? q2 : 0.0);
            __syncthreads();
            c = -m;
            if (r0 < 0.0)
                r0 = rn;
            if (rn <= rtol * r0)
                break;
            for (int colour = 0; colour < 2; ++colour) {
                const T *src = colour == 0 ? a : b;
                T *dst = colour == 0 ? b : a;
                if (mine) {
                    if (colour_me != colour) {
                        MG5_AT(dst, p) = MG5_AT(src, p);
                    } else {
                        St<T> s, sb;
                        gather_nbr(src, nb, s);
                        if constexpr (BASE)
                            gather_nbr(bs, nb, sb);
                        bool cl = false;
                        MG5_AT(dst, p) = upd<T, BASE>(s, sb, fme + (T)c, cf, cl);
                        my_clamps += cl ? 1ull : 0ull;
                    }
                }
                __syncthreads();
            }
        }
        nu_max = 0;   // skip the general loop
    }
    for (; it < nu_max; ++it) {
        double2 acc = make_double2(0.0, 0.0);
        for (int p = threadIdx.x; p < n3; p += blockDim.x) {
            const int k = p % n, j = (p / n) % n, i = p / (n * n);
            const Rows r = periodic_rows(n, i, j);
            const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
            St<T> s, sb;
            gather((const T *)a, (const T *)a, r, k, kp, km, s);
            if constexpr (BASE)
                gather(bs, bs, r, k, kp, km, sb);
            const double res = (double)resid_of<T, BASE>(s, sb, MG5_AT(ff, p), cf);
            acc.x += res;
            acc.y += res * res;
        }
        acc = block_sum2(acc);
        if (threadIdx.x == 0) {
            bc_s[0] = acc.x;
            bc_s[1] = acc.y;
        }
        __syncthreads();
        const double m = bc_s[0] * inv_n3;
        const double q2 = bc_s[1] - (double)n3 * m * m;
        const double rn = sqrt(q2 > 0.0 ? q2 : 0.0);
        __syncthreads();
        c = -m;
        if (r0 < 0.0)
            r0 = rn;
        if (rn <= rtol * r0)
            break;
        for (int colour = 0; colour < 2; ++colour) {
            const T *src = colour == 0 ? a : b;
            T *dst = colour == 0 ? b : a;
            for (int p = threadIdx.x; p < n3; p += blockDim.x) {
                const int k = p % n, j = (p / n) % n, i = p / (n * n);
                if (((i + j + k) & 1) != colour) {
                    MG5_AT(dst, p) = MG5_AT(src, p);
                    continue;
                }
                const Rows r = periodic_rows(n, i, j);
                const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
                St<T> s, sb;
                gather(src, src, r, k, kp, km, s);
                if constexpr (BASE)
                    gather(bs, bs, r, k, kp, km, sb);
                bool cl = false;
                MG5_AT(dst, p) = upd<T, BASE>(s, sb, MG5_AT(ff, p) + (T)c, cf, cl);
                my_clamps += cl ? 1ull : 0ull;
            }
            __syncthreads();
        }
    }
    if (in_smem)
        for (int p = threadIdx.x; p < n3; p += blockDim.x)
            MG5_AT(A, p) = MG5_AT(a, p);
    if (my_clamps)
        atomicAdd(&MG5_AT(clamp, 0), my_clamps);
    if (threadIdx.x == 0) {
        MG5_AT(cptr, 0) = c;
        if (sweeps_out)
            atomicAdd(&MG5_AT(sweeps_out, 0), it);
    }
}

template <typename T>
cudaError_t launch_coarsest(T *v, T *tmp, const T *f, int n, CoefT<T> cf, double *cptr, int nu_max,
                            double rtol, unsigned long long *clamp, int *sweeps, cudaStream_t st,
                            const T *B)
{
    const int n3 = n * n * n;
    int threads = ((n3 + 31) / 32) * 32;
    if (threads > kCoarsestThreads)
        threads = kCoarsestThreads;
    const size_t sm = n3 <= kCoarsestSmemCells ? (size_t)4 * n3 * sizeof(T) : 0;
    if (B)
        k_coarsest<T, true><<<1, threads, sm, st>>>(v, tmp, f, n, cf, cptr, nu_max, rtol, clamp,
                                                    sweeps, B);
    else
        k_coarsest<T, false><<<1, threads, sm, st>>>(v, tmp, f, n, cf, cptr, nu_max, rtol, clamp,
                                                     sweeps, B);
    count_launch(1);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// reductions
// --------------------------------------------------------------------------
__global__ void k_finalize(const double2 *__restrict__ partials, int nb, double ncells,
                           LevelScal *ls, int mode)
{
    finalize_body(partials, nb, ncells, ls, mode);
}

cudaError_t launch_finalize(const double2 *partials, int nb, double ncells, LevelScal *ls, int mode,
                            cudaStream_t st)
{
    k_finalize<<<1, 256, 0, st>>>(partials, nb, ncells, ls, mode);
    count_launch(1);
    return cudaGetLastError();
}

__global__ void k_scale(const double *__restrict__ delta, double s, double *__restrict__ f,
                        long long n3, double2 *__restrict__ partials, double add,
                        const double *__restrict__ add_dev, Fin fin)
{
    if (add_dev)
        add = *add_dev;
    double2 acc = make_double2(0.0, 0.0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n3;
         t += (long long)gridDim.x * blockDim.x) {
        const double v = s * MG5_AT(delta, t);
        MG5_AT(f, t) = v + add;
        acc.y += v * v;
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = acc;
    if (fin.ls)
        finalize_if_last(partials, fin);
}

cudaError_t launch_scale(const double *delta, double s, double *f, long long n3, double2 *partials,
                         int *nblocks, cudaStream_t st, double add, const double *add_dev,
                         const Fin &fin)
{
    int g = blocks_for(n3);
    if (g > kReduceBlocks)
        g = kReduceBlocks;
    k_scale<<<g, kBlock, 0, st>>>(delta, s, f, n3, partials, add, add_dev, fin);
    *nblocks = g;
    count_launch(1);
    return cudaGetLastError();
}

__global__ void k_sum(const double *__restrict__ a, long long n3, double2 *__restrict__ partials,
                      Fin fin)
{
    double2 acc = make_double2(0.0, 0.0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n3;
         t += (long long)gridDim.x * blockDim.x)
        acc.x += MG5_AT(a, t);
    acc = block_sum2(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = acc;
    if (fin.ls)
        finalize_if_last(partials, fin);
}

cudaError_t launch_sum(const double *phi, long long n3, double2 *partials, int *nblocks,
                       cudaStream_t st, const Fin &fin)
{
    int g = blocks_for(n3);
    if (g > kReduceBlocks)
        g = kReduceBlocks;
    k_sum<<<g, kBlock, 0, st>>>(phi, n3, partials, fin);
    *nblocks = g;
    count_launch(1);
    return cudaGetLastError();
}

__global__ void k_sub_mean(double *__restrict__ a, long long n3, const double *__restrict__ mean)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n3)
        MG5_AT(a, t) -= MG5_AT(mean, 0);
}

cudaError_t launch_sub_mean(double *phi, long long n3, const double *mean, cudaStream_t st)
{
    k_sub_mean<<<blocks_for(n3), kBlock, 0, st>>>(phi, n3, mean);
    count_launch(1);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// force: central differences at cell centres (Sec. 3.2), SoA output
// --------------------------------------------------------------------------
__global__ void k_force(const double *__restrict__ phi, int d0, int d1, int d2, int g, double inv2h,
                        int periodic, double *__restrict__ grad)
{
    const int n0 = d0 - 2 * g, n1 = d1 - 2 * g, n2 = d2 - 2 * g;
    const long long total = (long long)n0 * n1 * n2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int k = (int)(t % n2);
    const long long q = t / n2;
    const int j = (int)(q % n1), i = (int)(q / n1);
    const int I = i + g, J = j + g, K = k + g;
    int ip = I + 1, im = I - 1, jp = J + 1, jm = J - 1, kp = K + 1, km = K - 1;
    if (periodic) {
        ip = ip == d0 ? 0 : ip;
        im = im < 0 ? d0 - 1 : im;
        jp = jp == d1 ? 0 : jp;
        jm = jm < 0 ? d1 - 1 : jm;
        kp = kp == d2 ? 0 : kp;
        km = km < 0 ? d2 - 1 : km;
    }
    const long long D1 = d1, D2 = d2;
    auto at = [&](int a, int b, int c) { return MG5_AT(phi, ((long long)a * D1 + b) * D2 + c); };
    MG5_AT(grad, t) = (at(ip, J, K) - at(im, J, K)) * inv2h;
    MG5_AT(grad, total + t) = (at(I, jp, K) - at(I, jm, K)) * inv2h;
    MG5_AT(grad, 2 * total + t) = (at(I, J, kp) - at(I, J, km)) * inv2h;
}

cudaError_t launch_force(const double *phi, int d0, int d1, int d2, int ghost, double h, int periodic,
                         double *grad, cudaStream_t st)
{
    const long long work = (long long)(d0 - 2 * ghost) * (d1 - 2 * ghost) * (d2 - 2 * ghost);
    k_force<<<grid_spread(work), block_spread(work), 0, st>>>(phi, d0, d1, d2, ghost, 0.5 / h, periodic, grad);
    count_launch(1);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// coarse -> fine interpolation of phi (Sec. 3.1 / 3.2)
// fine local index I (ghosts included) -> coarse coordinate x = o + (I - g + 1/2)/2;
// t = x - 1/2 = o + (I - g)/2 - 1/4; i0 = floor(t), w = t - i0 in {1/4, 3/4}.
// --------------------------------------------------------------------------
// Source grid of the interpolation: a periodic cube (nc^3), or a box of dims c[3]
// whose interior starts at offset `pg` on every axis (no wrap; the caller checks
// that every stencil cell lies inside the box).
struct RefineSrc {
    int c0, c1, c2;   // dims of the stored array
    int pg;           // interior offset (0 for the periodic cube)
    int periodic;     // 1: wrap indices modulo c (cube)
};

__global__ void k_refine(const double *__restrict__ phic, RefineSrc src, int o0, int o1, int o2,
                         int d0, int d1, int d2, int g, double *__restrict__ fine)
{
    const long long total = (long long)d0 * d1 * d2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int K = (int)(t % d2);
    const long long q = t / d2;
    const int J = (int)(q % d1), I = (int)(q / d1);
    const int loc[3] = {I, J, K};
    const int org[3] = {o0, o1, o2};
    const int dim[3] = {src.c0, src.c1, src.c2};
    int lo[3], hi[3];
    double w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // 4 t = 4 o + 2 (I - g) - 1 is an exact integer
        const int t4 = 4 * org[a] + 2 * (loc[a] - g) - 1;
        const int i0 = (t4 >= 0) ? (t4 >> 2) : -((-t4 + 3) >> 2);
        w[a] = (double)(t4 - 4 * i0) * 0.25;
        if (src.periodic) {
            int l = i0 % dim[a];
            l = l < 0 ? l + dim[a] : l;
            lo[a] = l;
            hi[a] = (l + 1 == dim[a]) ? 0 : l + 1;
        } else {
            lo[a] = i0 + src.pg;
            hi[a] = i0 + 1 + src.pg;
        }
    }
    const long long C1 = src.c1, C2 = src.c2;
    double v = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const double wt = (a ? w[0] : 1.0 - w[0]) * (b ? w[1] : 1.0 - w[1]) *
                                  (c ? w[2] : 1.0 - w[2]);
                const long long idx =
                    ((long long)(a ? hi[0] : lo[0]) * C1 + (b ? hi[1] : lo[1])) * C2 +
                    (c ? hi[2] : lo[2]);
                v += wt * MG5_AT(phic, idx);
            }
    MG5_AT(fine, t) = v;
}

cudaError_t launch_refine(const double *phic, int nc, const int o[3], const int pn[3], int ghost,
                          double *fine, cudaStream_t st)
{
    const int d0 = 2 * pn[0] + 2 * ghost, d1 = 2 * pn[1] + 2 * ghost, d2 = 2 * pn[2] + 2 * ghost;
    const long long work = (long long)d0 * d1 * d2;
    const RefineSrc src{nc, nc, nc, 0, 1};
    k_refine<<<grid_spread(work), block_spread(work), 0, st>>>(phic, src, o[0], o[1], o[2], d0, d1, d2, ghost,
                                                  fine);
    count_launch(1);
    return cudaGetLastError();
}

// Tricubic variant (periodic source): per axis the fine centre sits a quarter cell right
// (w = 1/4) or three quarters right (w = 3/4) of coarse centre i0; the 4-point Lagrange
// weights on i0 - 1 .. i0 + 2 are then (-7, 105, 35, -5) / 128 or (-5, 35, 105, -7) / 128.
__global__ void k_refine_cubic(const double *__restrict__ phic, int nc, int o0, int o1, int o2,
                               int d0, int d1, int d2, int g, double *__restrict__ fine)
{
    const long long total = (long long)d0 * d1 * d2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int K = (int)(t % d2);
    const long long q = t / d2;
    const int J = (int)(q % d1), I = (int)(q / d1);
    const int loc[3] = {I, J, K};
    const int org[3] = {o0, o1, o2};
    int idx[3][4];
    double w[3][4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int t4 = 4 * org[a] + 2 * (loc[a] - g) - 1;   // 4 (coarse coordinate - 1/2)
        const int i0 = (t4 >= 0) ? (t4 >> 2) : -((-t4 + 3) >> 2);
        const bool quarter = (t4 - 4 * i0) == 1;
        w[a][0] = (quarter ? -7.0 : -5.0) / 128.0;
        w[a][1] = (quarter ? 105.0 : 35.0) / 128.0;
        w[a][2] = (quarter ? 35.0 : 105.0) / 128.0;
        w[a][3] = (quarter ? -5.0 : -7.0) / 128.0;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            int l = (i0 - 1 + m) % nc;
            idx[a][m] = l < 0 ? l + nc : l;
        }
    }
    const long long NC = nc;
    double v = 0.0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            const long long row = ((long long)idx[0][a] * NC + idx[1][b]) * NC;
            const double wab = w[0][a] * w[1][b];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                v += wab * w[2][c] * MG5_AT(phic, row + idx[2][c]);
        }
    MG5_AT(fine, t) = v;
}

cudaError_t launch_refine_cubic(const double *phic, int nc, const int o[3], const int pn[3], int ghost,
                                double *fine, cudaStream_t st)
{
    const int d0 = 2 * pn[0] + 2 * ghost, d1 = 2 * pn[1] + 2 * ghost, d2 = 2 * pn[2] + 2 * ghost;
    const long long work = (long long)d0 * d1 * d2;
    k_refine_cubic<<<grid_spread(work), block_spread(work), 0, st>>>(phic, nc, o[0], o[1], o[2], d0, d1, d2,
                                                        ghost, fine);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t launch_refine_box(const double *box, const int bd[3], int pg, const int o[3],
                              const int pn[3], int ghost, double *fine, cudaStream_t st)
{
    const int d0 = 2 * pn[0] + 2 * ghost, d1 = 2 * pn[1] + 2 * ghost, d2 = 2 * pn[2] + 2 * ghost;
    const long long work = (long long)d0 * d1 * d2;
    const RefineSrc src{bd[0], bd[1], bd[2], pg, 0};
    k_refine<<<grid_spread(work), block_spread(work), 0, st>>>(box, src, o[0], o[1], o[2], d0, d1, d2, ghost,
                                                  fine);
    count_launch(1);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Dirichlet patch: interior pf, box pf + 2, colour = parity of the interior index.
// --------------------------------------------------------------------------
// Coarse patch grids keep their ghosts on the extrapolated boundary condition
// g = v0(g) + w^m (v(a) - v0(a)) (k_patch.cu), where a is the one interior cell nearest g.
// The thread that writes interior cell a writes every ghost anchored at it, so the
// ghosts of `out` follow each half-sweep without a separate pass: the red pass writes the
// red cells and copies the black ones (except in the SPLIT form of k_patch_half), the black
// pass the relaxed black cells, and a ghost is only ever read by its own anchor's thread among
// the cells that write.
__device__ __forceinline__ void write_anchored_ghosts(double *dst, const double *__restrict__ v0,
                                                      double w, double val, int i, int j, int k,
                                                      int p0, int p1, int p2, int d1, int d2)
{
    // per axis: the cell's own box index, and the ghost planes below (index 0, when the cell
    // is the first interior one) and above (index p + 1, when it is the last) -- no arrays,
    // so nothing goes to local memory
    const bool li = i == 0, hi = i == p0 - 1, lj = j == 0, hj = j == p1 - 1, lk = k == 0,
               hk = k == p2 - 1;
    if (!(li | hi | lj | hj | lk | hk))
        return;
    const long long ab = ((long long)(i + 1) * d1 + (j + 1)) * d2 + (k + 1);
    const double da = val - MG5_AT(v0, ab);
    const int Iv[3] = {i + 1, 0, p0 + 1}, Jv[3] = {j + 1, 0, p1 + 1}, Kv[3] = {k + 1, 0, p2 + 1};
    const bool oi[3] = {true, li, hi}, oj[3] = {true, lj, hj}, ok[3] = {true, lk, hk};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int m = (a > 0) + (b > 0) + (c > 0);
                if (m == 0 || !(oi[a] && oj[b] && ok[c]))
                    continue;
                const double wm = m == 1 ? w : (m == 2 ? w * w : w * w * w);
                const long long g = ((long long)Iv[a] * d1 + Jv[b]) * d2 + Kv[c];
                MG5_AT(dst, g) = MG5_AT(v0, g) + wm * da;
            }
}

// One thread per pair of cells (k = 2m, 2m + 1) of a row: one of the two has the colour of
// the pass and is relaxed; with copy_other (the red pass) the other is carried into dst.
// SPLIT (unmasked coarse patch grids, whose half-sweeps are latency-bound): the red pass
// copies nothing, and the black pass reads what it would have copied (the old black values,
// and the ghosts anchored at black cells, rebuilt from them) from the sweep's input.  Every
// lane of a warp thus relaxes a cell (a thread per cell would leave half the lanes of each
// FP64 instruction idle, the colours alternating along k).  The sides are even on every grid
// the patch sweeps (the coarsest, possibly odd, is solved by k_pbox_coarsest).
// MASKED: interior cells with mask 0 are not relaxed (they keep their values).
// v0 (coarse patch grids): also refresh the ghosts anchored at the cells written.
template <bool MASKED, bool SPLIT>
__global__ void k_patch_half(const double *__restrict__ src_faces, const double *__restrict__ src_edges,
                             double *dst, const double *__restrict__ fint, double rhs_add, int p0,
                             int p1, int p2, CoefT<double> cf, int colour, int copy_other,
                             unsigned long long *clamp, const unsigned char *__restrict__ mask,
                             const double *__restrict__ v0, double w)
{
    const int h2 = p2 >> 1;
    const long long total = (long long)p0 * p1 * h2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int m = (int)(t % h2);
    const long long q = t / h2;
    const int j = (int)(q % p1), i = (int)(q / p1);
    const int d1 = p1 + 2, d2 = p2 + 2;
    const Rows r = box_rows(d1, d2, i + 1, j + 1);
    const int k = 2 * m + ((i + j + colour) & 1);   // (i + j + k) & 1 == colour
    const int K = k + 1;
    if (copy_other) {
        const int ko = k ^ 1;                        // the pair's cell of the other colour
        const double vo = MG5_AT(src_faces, r.r00 + ko + 1);
        MG5_AT(dst, r.r00 + ko + 1) = vo;
        if (v0)
            write_anchored_ghosts(dst, v0, w, vo, i, j, ko, p0, p1, p2, d1, d2);
    }
    const long long tk = ((long long)i * p1 + j) * p2 + k;
    if (MASKED && !MG5_AT(mask, tk)) {
        if (copy_other) {
            const double v = MG5_AT(src_faces, r.r00 + K);
            MG5_AT(dst, r.r00 + K) = v;
            if (v0)
                write_anchored_ghosts(dst, v0, w, v, i, j, k, p0, p1, p2, d1, d2);
        }
        return;
    }
    St<double> s;
    if (SPLIT && colour == 1) {
        // black pass after a red pass that copied nothing: the new red faces from src_faces;
        // the centre and the edges from src_edges, the sweep's input.  A face that is a ghost
        // is anchored at this cell: its boundary condition of the cell's input value,
        // v0(g) + w (v - v0(a)), is the value the red pass would have copied (the input's own
        // ghosts may predate a prolongation)
        gather3(src_faces, src_edges, src_edges, r, K, K + 1, K - 1, s);
        const bool gxm = i == 0, gxp = i == p0 - 1, gym = j == 0, gyp = j == p1 - 1, gzm = k == 0,
                   gzp = k == p2 - 1;
        if (gxm | gxp | gym | gyp | gzm | gzp) {
            const double da = s.c - MG5_AT(v0, r.r00 + K);
            const auto bc = [&](long long g) { return MG5_AT(v0, g) + w * da; };
            if (gxm)
                s.xm = bc(r.rm0 + K);
            if (gxp)
                s.xp = bc(r.rp0 + K);
            if (gym)
                s.ym = bc(r.r0m + K);
            if (gyp)
                s.yp = bc(r.r0p + K);
            if (gzm)
                s.zm = bc(r.r00 + K - 1);
            if (gzp)
                s.zp = bc(r.r00 + K + 1);
        }
    } else {
        gather(src_faces, src_edges, r, K, K + 1, K - 1, s);
    }
    bool cl = false;
    const double v = cell_update(s, MG5_AT(fint, tk) + rhs_add, cf, cl);
    MG5_AT(dst, r.r00 + K) = v;
    if (v0)
        write_anchored_ghosts(dst, v0, w, v, i, j, k, p0, p1, p2, d1, d2);
    if (cl)
        atomicAdd(&MG5_AT(clamp, 0), 1ull);
}

cudaError_t launch_patch_sweep(const double *in, double *out, const double *fint, double rhs_add,
                               const int pf[3], CoefT<double> cf, unsigned long long *clamp,
                               cudaStream_t st, const double *v0, double w,
                               const unsigned char *mask)
{
    if ((pf[0] | pf[1] | pf[2]) & 1)
        return cudaErrorInvalidValue;   // the pair mapping needs even sides
    const long long work = (long long)pf[0] * pf[1] * (pf[2] / 2);
    const int bs = block_spread(work), g = grid_spread(work);
    const bool split = !mask && v0;
    auto half = [&](const double *faces, int colour, int copy_other) {
        if (mask)
            k_patch_half<true, false><<<g, bs, 0, st>>>(faces, in, out, fint, rhs_add, pf[0],
                                                        pf[1], pf[2], cf, colour, copy_other, clamp,
                                                        mask, v0, w);
        else if (split)
            k_patch_half<false, true><<<g, bs, 0, st>>>(faces, in, out, fint, rhs_add, pf[0],
                                                        pf[1], pf[2], cf, colour, copy_other, clamp,
                                                        mask, v0, w);
        else
            k_patch_half<false, false><<<g, bs, 0, st>>>(faces, in, out, fint, rhs_add, pf[0],
                                                         pf[1], pf[2], cf, colour, copy_other,
                                                         clamp, mask, v0, w);
    };
    // red: from in, the black cells carried into out (SPLIT: not carried); black: faces from
    // out (new red), edges from in (old black), SPLIT: the centre and the ghost faces too
    half(in, 0, split ? 0 : 1);
    half(out, 1, 0);
    count_launch(2);
    return cudaGetLastError();
}

template <bool MASKED>
__global__ void k_patch_residual(const double *__restrict__ phi, const double *__restrict__ fint,
                                 double rhs_add, int p0, int p1, int p2, CoefT<double> cf,
                                 double2 *__restrict__ partials, const unsigned char *__restrict__ mask,
                                 Fin fin)
{
    const long long total = (long long)p0 * p1 * p2;
    double2 acc = make_double2(0.0, 0.0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        if (MASKED && !MG5_AT(mask, t))
            continue;
        const int k = (int)(t % p2);
        const long long q = t / p2;
        const int j = (int)(q % p1), i = (int)(q / p1);
        const Rows r = box_rows(p1 + 2, p2 + 2, i + 1, j + 1);
        St<double> s;
        gather(phi, phi, r, k + 1, k + 2, k, s);
        const double res = cell_residual(s, MG5_AT(fint, t) + rhs_add, cf);
        acc.x += res;
        acc.y += res * res;
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = acc;
    if (fin.ls)
        finalize_if_last(partials, fin);
}

cudaError_t launch_patch_residual(const double *phi, const double *fint, double rhs_add,
                                  const int pf[3], CoefT<double> cf, double2 *partials, int *nblocks,
                                  cudaStream_t st, const unsigned char *mask,
                                  const Fin &fin)
{
    const long long work = (long long)pf[0] * pf[1] * pf[2];
    const int bs = block_spread(work);
    int g = grid_spread(work);
    if (g > kReduceBlocksFp64)
        g = kReduceBlocksFp64;
    if (mask)
        k_patch_residual<true><<<g, bs, 0, st>>>(phi, fint, rhs_add, pf[0], pf[1], pf[2], cf,
                                                     partials, mask, fin);
    else
        k_patch_residual<false><<<g, bs, 0, st>>>(phi, fint, rhs_add, pf[0], pf[1], pf[2], cf,
                                                      partials, mask, fin);
    *nblocks = g;
    count_launch(1);
    return cudaGetLastError();
}

// explicit instantiations
#define MG5_INST(T)                                                                                \
    template cudaError_t launch_sweep<T>(const T *, T *, const T *, const double *, int, CoefT<T>, \
                                         unsigned long long *, cudaStream_t, const T *, int);      \
    template cudaError_t launch_operator<T>(const T *, int, CoefT<T>, T *, cudaStream_t);          \
    template cudaError_t launch_residual<T>(const T *, const T *, const double *, int, CoefT<T>,   \
                                            T *, double2 *, int *, cudaStream_t, const Fin &);     \
    template cudaError_t launch_resid_restrict<T>(const T *, const T *, const double *, int,       \
                                                  CoefT<T>, T *, T *, T *, double2 *, int *,       \
                                                  cudaStream_t, const T *, const Fin &);           \
    template cudaError_t launch_restrict<T>(const T *, int, T *, cudaStream_t);                    \
    template cudaError_t launch_coarse_rhs<T>(const T *, T *, const double *, double *, int,       \
                                              CoefT<T>, cudaStream_t, const T *);                  \
    template cudaError_t launch_prolong_add<T>(const T *, const T *, int, T *, double *,           \
                                               const double *, cudaStream_t);                      \
    template cudaError_t launch_coarsest<T>(T *, T *, const T *, int, CoefT<T>, double *, int,     \
                                            double, unsigned long long *, int *, cudaStream_t,     \
                                            const T *);
MG5_INST(double)
MG5_INST(float)

}  // namespace mg5
