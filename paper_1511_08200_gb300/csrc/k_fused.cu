// k_fused.cu -- fused red+black snapshot sweep: one kernel reads phi once and
// writes it once per full sweep.
//
// A CTA owns a TJ x TK tile of (j, k) and marches along i over a chunk of
// planes, keeping rings of planes in shared memory:
//   old  : planes p-1 .. p+2 of the input, tile + 2 halo (snapshot values),
//   base : the same planes of the correction base B (mixed precision only),
//   rnew : planes p-1 .. p+1 of the new red values, tile + 1 halo.
// At plane p it first relaxes the red cells of plane p+1 (tile + 1 halo, from
// `old`), then the black cells of plane p (faces from `rnew`, edges from
// `old`), and writes both colours of plane p.  Every read of a same-colour
// neighbour therefore sees the value from before its half-sweep, which is the
// snapshot red-black sweep the oracle defines; the red halo is recomputed by
// neighbouring tiles instead of exchanged.  Out of place: `in` and `out` must
// not alias.  Periodic in i, j, k.
#include "mg5_kernels.cuh"

namespace mg5 {

constexpr int FT_K = 32;           // tile along k (one warp)
constexpr int FT_J = 16;           // tile along j
constexpr int FT_THREADS = 256;
constexpr int OK_ = FT_K + 4;      // old/base plane row length
constexpr int OJ_ = FT_J + 4;
constexpr int RK_ = FT_K + 2;      // rnew plane row length
constexpr int RJ_ = FT_J + 2;
constexpr int OPL = OJ_ * OK_;     // elements of one old plane
constexpr int RPL = RJ_ * RK_;

template <typename T, bool BASE>
struct FusedSmem {
    T old[4][OPL];
    T base[BASE ? 4 : 1][BASE ? OPL : 1];
    T rnew[3][RPL];
};

template <typename T>
__device__ __forceinline__ void load_plane(T *dst, const T *__restrict__ src, int n, int i, int j0,
                                           int k0)
{
    const int ii = i < 0 ? i + n : (i >= n ? i - n : i);
    const long long pbase = (long long)ii * n * n;
    for (int e = threadIdx.x; e < OPL; e += FT_THREADS) {
        const int jj = e / OK_, kk = e - jj * OK_;
        int j = j0 - 2 + jj, k = k0 - 2 + kk;
        j = ((j % n) + n) % n;
        k = ((k % n) + n) % n;
        dst[e] = src[pbase + (long long)j * n + k];
    }
}

// gather the 19-point stencil around old-plane coordinates (jj, kk) of plane slot m
template <typename T>
__device__ __forceinline__ void gather_old(const T *pm, const T *p0, const T *pp, int jj, int kk,
                                           St<T> &s)
{
    const int c = jj * OK_ + kk;
    s.c = p0[c];
    s.xp = pp[c];
    s.xm = pm[c];
    s.yp = p0[c + OK_];
    s.ym = p0[c - OK_];
    s.zp = p0[c + 1];
    s.zm = p0[c - 1];
    s.xpyp = pp[c + OK_];
    s.xpym = pp[c - OK_];
    s.xmyp = pm[c + OK_];
    s.xmym = pm[c - OK_];
    s.xpzp = pp[c + 1];
    s.xpzm = pp[c - 1];
    s.xmzp = pm[c + 1];
    s.xmzm = pm[c - 1];
    s.ypzp = p0[c + OK_ + 1];
    s.ypzm = p0[c + OK_ - 1];
    s.ymzp = p0[c - OK_ + 1];
    s.ymzm = p0[c - OK_ - 1];
}

template <typename T, bool BASE>
__global__ void __launch_bounds__(FT_THREADS)
    k_sweep_fused(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ f,
                  const T *__restrict__ B, const double *__restrict__ cptr, int n, int ichunk,
                  CoefT<T> cf, unsigned long long *clamp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<T, BASE> &S = *reinterpret_cast<FusedSmem<T, BASE> *>(smem_raw);
    const int k0 = blockIdx.x * FT_K, j0 = blockIdx.y * FT_J;
    const int i0 = blockIdx.z * ichunk;
    const int i1 = min(i0 + ichunk, n);
    const T cval = (T)(*cptr);
    bool clamped = false;

    // relax the red cells of plane q on the tile + 1 halo into rnew[slot]
    auto red_plane = [&](int q) {
        const int sm = ((q - 1) % 4 + 4) % 4, s0 = ((q % 4) + 4) % 4, sp = ((q + 1) % 4 + 4) % 4;
        T *rn = S.rnew[((q % 3) + 3) % 3];
        const int qq = q < 0 ? q + n : (q >= n ? q - n : q);
        for (int e = threadIdx.x; e < RJ_ * (RK_ / 2); e += FT_THREADS) {
            const int jj = e / (RK_ / 2), pr = e - jj * (RK_ / 2);
            // red: (q + j + k) even with j = j0 - 1 + jj, k = k0 - 1 + kk
            const int kk = 2 * pr + ((q + j0 + jj + k0) & 1);
            int j = j0 - 1 + jj, k = k0 - 1 + kk;
            j = ((j % n) + n) % n;
            k = ((k % n) + n) % n;
            St<T> s, sb;
            gather_old(S.old[sm], S.old[s0], S.old[sp], jj + 1, kk + 1, s);
            if constexpr (BASE)
                gather_old(S.base[sm], S.base[s0], S.base[sp], jj + 1, kk + 1, sb);
            const T rhs = f[((long long)qq * n + j) * n + k] + cval;
            rn[jj * RK_ + kk] = upd<T, BASE>(s, sb, rhs, cf, clamped);
        }
    };

    // prologue: old planes i0-2 .. i0+1, red planes i0-1 and i0
    for (int q = i0 - 2; q <= i0 + 1; ++q) {
        load_plane(S.old[((q % 4) + 4) % 4], in, n, q, j0, k0);
        if constexpr (BASE)
            load_plane(S.base[((q % 4) + 4) % 4], B, n, q, j0, k0);
    }
    __syncthreads();
    red_plane(i0 - 1);
    red_plane(i0);

    for (int p = i0; p < i1; ++p) {
        __syncthreads();  // the slot of plane p-2 is free: black(p-1) has finished
        load_plane(S.old[((p + 2) % 4)], in, n, p + 2, j0, k0);
        if constexpr (BASE)
            load_plane(S.base[((p + 2) % 4)], B, n, p + 2, j0, k0);
        __syncthreads();
        red_plane(p + 1);
        __syncthreads();
        // black cells of plane p over the tile; each thread owns the pair (2 pr, 2 pr + 1)
        {
            const int jj = threadIdx.x / (FT_K / 2), pr = threadIdx.x - jj * (FT_K / 2);
            const int j = j0 + jj, kp0 = k0 + 2 * pr;
            const int bodd = (p + j + kp0 + 1) & 1;  // 0: black is the first of the pair
            const int kk = 2 * pr + bodd;            // tile-local k of the black cell
            const T *om = S.old[(p + 3) % 4], *o0 = S.old[p % 4], *op = S.old[(p + 1) % 4];
            const T *rm = S.rnew[(p + 2) % 3], *r0 = S.rnew[p % 3], *rp = S.rnew[(p + 1) % 3];
            // faces (red, new) from rnew; edges (black, old) from old
            const int cr = (jj + 1) * RK_ + (kk + 1);
            const int co = (jj + 2) * OK_ + (kk + 2);
            St<T> s;
            s.c = o0[co];
            s.xp = rp[cr];
            s.xm = rm[cr];
            s.yp = r0[cr + RK_];
            s.ym = r0[cr - RK_];
            s.zp = r0[cr + 1];
            s.zm = r0[cr - 1];
            s.xpyp = op[co + OK_];
            s.xpym = op[co - OK_];
            s.xmyp = om[co + OK_];
            s.xmym = om[co - OK_];
            s.xpzp = op[co + 1];
            s.xpzm = op[co - 1];
            s.xmzp = om[co + 1];
            s.xmzm = om[co - 1];
            s.ypzp = o0[co + OK_ + 1];
            s.ypzm = o0[co + OK_ - 1];
            s.ymzp = o0[co - OK_ + 1];
            s.ymzm = o0[co - OK_ - 1];
            St<T> sb;
            if constexpr (BASE)
                gather_old(S.base[(p + 3) % 4], S.base[p % 4], S.base[(p + 1) % 4], jj + 2, kk + 2, sb);
            if (j < n && kp0 < n) {
                const long long row = ((long long)p * n + j) * n;
                const T vb = upd<T, BASE>(s, sb, f[row + k0 + kk] + cval, cf, clamped);
                const T vr = r0[(jj + 1) * RK_ + (2 * pr + 1 - bodd) + 1];
                T v0 = bodd ? vr : vb;
                T v1 = bodd ? vb : vr;
                if constexpr (sizeof(T) == 4) {
                    float2 w;
                    w.x = (float)v0;
                    w.y = (float)v1;
                    *reinterpret_cast<float2 *>(out + row + kp0) = w;
                } else {
                    double2 w;
                    w.x = (double)v0;
                    w.y = (double)v1;
                    *reinterpret_cast<double2 *>(out + row + kp0) = w;
                }
            }
        }
    }
    if (clamped)
        atomicAdd(clamp, 1ull);
}

template <typename T>
cudaError_t launch_sweep_fused(const T *in, T *out, const T *f, const double *cptr, int n,
                               CoefT<T> cf, unsigned long long *clamp, cudaStream_t st, const T *B)
{
    const int tk = (n + FT_K - 1) / FT_K, tj = (n + FT_J - 1) / FT_J;
    const int tiles = tk * tj;
    // enough CTAs to fill 152 SMs several times over, chunks of at least 8 planes
    int chunks = (4 * 152 + tiles - 1) / tiles;
    if (chunks > n / 8)
        chunks = n / 8;
    if (chunks < 1)
        chunks = 1;
    const int ichunk = (n + chunks - 1) / chunks;
    chunks = (n + ichunk - 1) / ichunk;
    dim3 grid(tk, tj, chunks);
    cudaError_t e;
    if (B) {
        const size_t sm = sizeof(FusedSmem<T, true>);
        e = cudaFuncSetAttribute(k_sweep_fused<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess)
            return e;
        k_sweep_fused<T, true><<<grid, FT_THREADS, sm, st>>>(in, out, f, B, cptr, n, ichunk, cf, clamp);
    } else {
        const size_t sm = sizeof(FusedSmem<T, false>);
        e = cudaFuncSetAttribute(k_sweep_fused<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm);
        if (e != cudaSuccess)
            return e;
        k_sweep_fused<T, false><<<grid, FT_THREADS, sm, st>>>(in, out, f, B, cptr, n, ichunk, cf, clamp);
    }
    count_launch(1);
    return cudaGetLastError();
}

template cudaError_t launch_sweep_fused<float>(const float *, float *, const float *, const double *,
                                               int, CoefT<float>, unsigned long long *, cudaStream_t,
                                               const float *);
template cudaError_t launch_sweep_fused<double>(const double *, double *, const double *,
                                                const double *, int, CoefT<double>,
                                                unsigned long long *, cudaStream_t, const double *);

}  // namespace mg5
