// k_spectral.cu -- coarsest-grid solve for periodic coarsest grids of more than 6^3 cells.
//
// A grid side N = 2^a m with m odd stops halving at 2m (the 8-child restriction needs
// even sides), so N = 144, 176, 208, 240 end on coarsest grids of 18^3 .. 30^3 where
// Gauss-Seidel alone needs hundreds of sweeps to reduce the residual 1e-3 (the coarsest
// solve of Sec. 3.1's multigrid).  Here each iteration computes the residual
// r = f + c - op(v) (c = minus its mean, the compatibility constant), solves L d = r for
// the periodic 7-point Laplacian exactly -- separable discrete Fourier transforms, d_hat =
// r_hat / lambda(k), the mean mode dropped -- adds d to v, and smooths with two red-black
// sweeps.  L is the linear part of the operator, so the correction removes the smooth
// error the sweeps cannot, and the sweeps the local nonlinear part.  A fixed number of
// iterations keeps the launch sequence fixed (the same in captured graphs).  Multi-CTA
// kernels: the grid is at most 32^3.
#include "mg5_fin.cuh"

namespace mg5 {

template <typename T>
struct Cplx;
template <>
struct Cplx<double> {
    using type = double2;
};
template <>
struct Cplx<float> {
    using type = float2;
};

__device__ __forceinline__ void sincos_pi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ void sincos_pi(float x, float *s, float *c) { sincospif(x, s, c); }

// r = f + c - op(v) into the real parts (imaginary parts 0); block partial sums of (r, r^2);
// each call counts the two sweeps of its iteration.
template <typename T, bool BASE>
__global__ void k_spec_residual(const T *__restrict__ v, const T *__restrict__ f,
                                const double *__restrict__ cptr, int n, CoefT<T> cf,
                                const T *__restrict__ B, typename Cplx<T>::type *__restrict__ out,
                                Moments *__restrict__ partials, int *sweeps, Fin fin)
{
    const int n3 = n * n * n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    MomAcc<T> acc;
    if (t < n3) {
        const int k = t % n, j = (t / n) % n, i = t / (n * n);
        const Rows r = periodic_rows(n, i, j);
        const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
        St<T> s, sb;
        gather(v, v, r, k, kp, km, s);
        if constexpr (BASE)
            gather(B, B, r, k, kp, km, sb);
        const T res = resid_of<T, BASE>(s, sb, MG5_AT(f, t) + (T)(MG5_AT(cptr, 0)), cf);
        MG5_AT(out, t).x = res;
        MG5_AT(out, t).y = (T)0;
        acc.add(res);
    }
    const Moments m = block_moments(acc);
    if (threadIdx.x == 0) {
        MG5_AT(partials, blockIdx.x) = m;
        if (blockIdx.x == 0 && sweeps)
            atomicAdd(&MG5_AT(sweeps, 0), 2);
    }
    finalize_if_last(reinterpret_cast<double2 *>(partials), fin);   // c -= mean r
}

// One-dimensional DFT along `axis` (0: i, 1: j, 2: k) of every line:
// out[m'] = sum_m in[m] exp(-+ 2 pi i m m' / n) (sign: forward -, inverse +).  With `addto`,
// the real part times `scale` is added to it instead of writing `out`.
template <typename T>
__global__ void k_dft_axis(const typename Cplx<T>::type *__restrict__ in,
                           typename Cplx<T>::type *__restrict__ out, int n, int axis, int inverse,
                           T *__restrict__ addto, T scale)
{
    const int n3 = n * n * n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3)
        return;
    const int k = t % n, j = (t / n) % n, i = t / (n * n);
    const int mo = axis == 0 ? i : (axis == 1 ? j : k);
    const int stride = axis == 0 ? n * n : (axis == 1 ? n : 1);
    const int base = t - mo * stride;
    const T sgn = inverse ? (T)1 : (T)-1;
    T re = 0, im = 0;
    for (int m = 0; m < n; ++m) {
        const int q = (m * mo) % n;
        T sn, cs;
        sincos_pi((T)(2 * q) / (T)n, &sn, &cs);
        sn *= sgn;
        const typename Cplx<T>::type a = MG5_AT(in, base + m * stride);
        re += a.x * cs - a.y * sn;
        im += a.x * sn + a.y * cs;
    }
    if (addto) {
        MG5_AT(addto, t) += re * scale;
    } else {
        MG5_AT(out, t).x = re;
        MG5_AT(out, t).y = im;
    }
}

// d_hat = r_hat / lambda(k), lambda = (2 cos 2 pi kx/n + 2 cos 2 pi ky/n + 2 cos 2 pi kz/n - 6) / h^2
// (the periodic 7-point Laplacian's eigenvalue); the mean mode is set to zero.
template <typename T>
__global__ void k_spec_divide(typename Cplx<T>::type *__restrict__ a, int n, T h2)
{
    const int n3 = n * n * n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3)
        return;
    const int k = t % n, j = (t / n) % n, i = t / (n * n);
    if (i == 0 && j == 0 && k == 0) {
        MG5_AT(a, t).x = (T)0;
        MG5_AT(a, t).y = (T)0;
        return;
    }
    T s, ci, cj, ck;
    sincos_pi((T)(2 * i) / (T)n, &s, &ci);
    sincos_pi((T)(2 * j) / (T)n, &s, &cj);
    sincos_pi((T)(2 * k) / (T)n, &s, &ck);
    const T inv = h2 / ((T)2 * (ci + cj + ck) - (T)6);
    MG5_AT(a, t).x *= inv;
    MG5_AT(a, t).y *= inv;
}

template <typename T>
cudaError_t launch_coarsest_spectral(T *v, T *tmp, const T *f, int n, CoefT<T> cf, LevelScal *ls,
                                     int iters, unsigned long long *clamp, int *sweeps,
                                     double2 *partials, void *w0v, void *w1v, cudaStream_t st,
                                     const T *B)
{
    using C = typename Cplx<T>::type;
    C *w0 = static_cast<C *>(w0v), *w1 = static_cast<C *>(w1v);
    const int n3 = n * n * n;
    const int g = (n3 + kBlock - 1) / kBlock;
    if (g > kMomentBlocks)
        return cudaErrorInvalidValue;
    Moments *mp = reinterpret_cast<Moments *>(partials);
    const T inv_n3 = (T)1 / (T)n3;
    for (int it = 0; it < iters; ++it) {
        const Fin fin{ls, FIN_RESID, (double)n3};
        if (B)
            k_spec_residual<T, true><<<g, kBlock, 0, st>>>(v, f, &ls->c, n, cf, B, w0, mp, sweeps, fin);
        else
            k_spec_residual<T, false><<<g, kBlock, 0, st>>>(v, f, &ls->c, n, cf, B, w0, mp, sweeps, fin);
        count_launch(1);
        cudaError_t e;
        k_dft_axis<T><<<g, kBlock, 0, st>>>(w0, w1, n, 2, 0, nullptr, (T)0);
        k_dft_axis<T><<<g, kBlock, 0, st>>>(w1, w0, n, 1, 0, nullptr, (T)0);
        k_dft_axis<T><<<g, kBlock, 0, st>>>(w0, w1, n, 0, 0, nullptr, (T)0);
        k_spec_divide<T><<<g, kBlock, 0, st>>>(w1, n, cf.h2);
        k_dft_axis<T><<<g, kBlock, 0, st>>>(w1, w0, n, 0, 1, nullptr, (T)0);
        k_dft_axis<T><<<g, kBlock, 0, st>>>(w0, w1, n, 1, 1, nullptr, (T)0);
        k_dft_axis<T><<<g, kBlock, 0, st>>>(w1, w0, n, 2, 1, v, inv_n3);   // v += Re(d)
        count_launch(7);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        e = launch_sweep<T>(v, tmp, f, &ls->c, n, cf, clamp, st, B);
        if (e == cudaSuccess)
            e = launch_sweep<T>(tmp, v, f, &ls->c, n, cf, clamp, st, B);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

template cudaError_t launch_coarsest_spectral<double>(double *, double *, const double *, int,
                                                      CoefT<double>, LevelScal *, int,
                                                      unsigned long long *, int *, double2 *, void *,
                                                      void *, cudaStream_t, const double *);
template cudaError_t launch_coarsest_spectral<float>(float *, float *, const float *, int,
                                                     CoefT<float>, LevelScal *, int,
                                                     unsigned long long *, int *, double2 *, void *,
                                                     void *, cudaStream_t, const float *);

}  // namespace mg5
