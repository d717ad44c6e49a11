// k_fused.cu -- fused red+black snapshot sweep: one kernel reads phi once and
// writes it once per full sweep.
//
// A CTA owns a TJ x TK tile of (j, k) and marches along i over a chunk of
// planes, keeping rings of planes in shared memory:
//   old  : planes p-1 .. p+3 of the input, tile + 2 halo (snapshot values),
//   fr   : the same planes of the right-hand side f,
//   base : the same planes of the correction base B (mixed precision only),
//   rnew : planes p-1 .. p+1 of the new red values, tile + 1 halo.
// At plane p it relaxes the red cells of plane p+1 (tile + 1 halo, from
// `old`), then the black cells of plane p (faces from `rnew`, edges from
// `old`), and writes both colours of plane p, while plane p+3 streams into
// shared memory with cp.async.  Every read of a same-colour neighbour sees
// the value from before its half-sweep: the snapshot red-black sweep the
// oracle defines.  The red halo is recomputed by neighbouring tiles instead
// of exchanged.  Out of place (`in` and `out` must not alias); periodic in
// i, j, k; n must be a multiple of 16 / sizeof(T) (16-byte row chunks).
#include "mg5_kernels.cuh"

namespace mg5 {

constexpr int FT_K = 32;                // tile along k
constexpr int FT_J = 16;                // tile along j
constexpr int FT_THREADS = 320;         // 306 red cells of the halo'd plane in one round
constexpr int OROW = FT_K + 8;          // old/base row: k0 - 4 .. k0 + 35 (16-byte chunks)
constexpr int OJ_ = FT_J + 4;           // rows j0 - 2 .. j0 + 17
constexpr int OPL = OJ_ * OROW;         // elements of one old plane
constexpr int RK_ = FT_K + 2;           // rnew row: k0 - 1 .. k0 + 32
constexpr int RJ_ = FT_J + 2;
constexpr int RPL = RJ_ * RK_;
constexpr int NSLOT = 5;                // planes p-1 .. p+3

template <typename T, bool BASE>
struct FusedSmem {
    T old[NSLOT][OPL];
    T fr[NSLOT][OPL];                       // right-hand side planes, same layout
    T base[BASE ? NSLOT : 1][BASE ? OPL : 1];
    T rnew[3][RPL];
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
#ifdef MG5_BOUNDS
    if (!::mg5::bnd::copy_ok(s, gmem, __LINE__))
        return;
#endif
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int wrap1(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }
__device__ __forceinline__ int slot5(int q) { return ((q % NSLOT) + NSLOT) % NSLOT; }

// Ring slots of planes q-1, q, q+1 (q >= -2 here): one unsigned division, then increments.
struct Ring {
    int m, z, p;
};
template <int K>
__device__ __forceinline__ Ring ring(int q)
{
    const int m = (int)((unsigned)(q - 1 + 3 * K) % (unsigned)K);
    const int z = m == K - 1 ? 0 : m + 1;
    return Ring{m, z, z == K - 1 ? 0 : z + 1};
}

// The 16-byte copies of one plane (rows j0-2 .. j0+17, k0-4 .. k0+35) that this thread
// issues: the same (row, chunk) positions for every plane and array, so their shared and
// global offsets within a plane are computed once per CTA.
template <typename T>
struct CopyPlan {
    static constexpr int EPC = 16 / sizeof(T);                  // elements per chunk
    static constexpr int CPR = OROW / EPC;                      // chunks per row
    static constexpr int NCH = OJ_ * CPR;                       // chunks per plane
    static constexpr int PER = (NCH + FT_THREADS - 1) / FT_THREADS;
    int soff[PER];   // shared offset within a plane
    int goff[PER];   // global offset within a plane (j n + k); -1: no chunk
};

template <typename T>
__device__ __forceinline__ CopyPlan<T> make_plan(int n, int j0, int k0)
{
    CopyPlan<T> pl;
#pragma unroll
    for (int m = 0; m < CopyPlan<T>::PER; ++m) {
        const int c = threadIdx.x + m * FT_THREADS;
        pl.goff[m] = -1;
        pl.soff[m] = 0;
        if (c < CopyPlan<T>::NCH) {
            const int r = c / CopyPlan<T>::CPR, cc = c - r * CopyPlan<T>::CPR;
            const int j = wrap1(j0 - 2 + r, n);
            const int k = wrap1(k0 - 4 + cc * CopyPlan<T>::EPC, n);
            pl.soff[m] = r * OROW + cc * CopyPlan<T>::EPC;
            pl.goff[m] = j * n + k;
        }
    }
    return pl;
}

// issue this thread's copies of the plane that starts at global offset pb
template <typename T>
__device__ __forceinline__ void issue_plane(T *dst, const T *__restrict__ src, long long pb,
                                            const CopyPlan<T> &pl)
{
#pragma unroll
    for (int m = 0; m < CopyPlan<T>::PER; ++m)
        if (pl.goff[m] >= 0)
            cp_async16(dst + pl.soff[m], src + pb + pl.goff[m]);
}

// 19-point stencil around old-plane row jr, column kc
template <typename T>
__device__ __forceinline__ void gather_old(const T *pm, const T *p0, const T *pp, int jr, int kc,
                                           St<T> &s)
{
    const int c = jr * OROW + kc;
    s.c = MG5_AT(p0, c);
    s.xp = MG5_AT(pp, c);
    s.xm = MG5_AT(pm, c);
    s.yp = MG5_AT(p0, c + OROW);
    s.ym = MG5_AT(p0, c - OROW);
    s.zp = MG5_AT(p0, c + 1);
    s.zm = MG5_AT(p0, c - 1);
    s.xpyp = MG5_AT(pp, c + OROW);
    s.xpym = MG5_AT(pp, c - OROW);
    s.xmyp = MG5_AT(pm, c + OROW);
    s.xmym = MG5_AT(pm, c - OROW);
    s.xpzp = MG5_AT(pp, c + 1);
    s.xpzm = MG5_AT(pp, c - 1);
    s.xmzp = MG5_AT(pm, c + 1);
    s.xmzm = MG5_AT(pm, c - 1);
    s.ypzp = MG5_AT(p0, c + OROW + 1);
    s.ypzm = MG5_AT(p0, c + OROW - 1);
    s.ymzp = MG5_AT(p0, c - OROW + 1);
    s.ymzm = MG5_AT(p0, c - OROW - 1);
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
    const T cval = (T)(MG5_AT(cptr, 0));
    bool clamped = false;
    const CopyPlan<T> plan = make_plan<T>(n, j0, k0);
    const long long n2 = (long long)n * n;
    auto plane_at = [&](int q) { return (long long)wrap1(q, n) * n2; };

    // red cells of plane q on the tile + 1 halo -> rnew[slot3(q)]
    auto red_plane = [&](int q) {
        const Ring r5 = ring<NSLOT>(q);
        const T *om = S.old[r5.m], *o0 = S.old[r5.z], *op = S.old[r5.p];
        T *rn = S.rnew[ring<3>(q).z];
        // rows of 16 pairs per half-warp (a half-warp's cells sit in one row, 2 apart;
        // the two halves of a warp take rows of opposite parity, so with even row
        // strides the 32 lanes hit 32 distinct banks), then the 17th pair of each row
        const int e = threadIdx.x;
        if (e < RJ_ * (RK_ / 2)) {
            const int main_n = RJ_ * 16;
            const int jj = e < main_n ? e >> 4 : e - main_n;
            const int pr = e < main_n ? (e & 15) : 16;
            // red: (q + j + k) even, j = j0 - 1 + jj, k = k0 - 1 + kk
            const int kk = 2 * pr + ((q + j0 + jj + k0) & 1);
            St<T> s, sb;
            gather_old(om, o0, op, jj + 1, kk + 3, s);
            if constexpr (BASE)
                gather_old(S.base[r5.m], S.base[r5.z], S.base[r5.p], jj + 1, kk + 3, sb);
            const T rhs = S.fr[r5.z][(jj + 1) * OROW + kk + 3] + cval;
            MG5_AT(rn, jj * RK_ + kk) = upd<T, BASE>(s, sb, rhs, cf, clamped);
        }
    };

    // prologue: planes i0-2 .. i0+1 (group 1), plane i0+2 (group 2)
    for (int q = i0 - 2; q <= i0 + 1; ++q) {
        const long long pb = plane_at(q);
        issue_plane(S.old[slot5(q)], in, pb, plan);
        if (q >= i0 - 1)
            issue_plane(S.fr[slot5(q)], f, pb, plan);
        if constexpr (BASE)
            issue_plane(S.base[slot5(q)], B, pb, plan);
    }
    cp_async_commit();
    {
        const long long pb = plane_at(i0 + 2);
        issue_plane(S.old[slot5(i0 + 2)], in, pb, plan);
        issue_plane(S.fr[slot5(i0 + 2)], f, pb, plan);
        if constexpr (BASE)
            issue_plane(S.base[slot5(i0 + 2)], B, pb, plan);
    }
    cp_async_commit();
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    red_plane(i0 - 1);
    red_plane(i0);

    for (int p = i0; p < i1; ++p) {
        cp_async_wait_all();   // plane p+2 has landed
        __syncthreads();       // ... for every thread; iteration p-1 is finished everywhere
        {
            const long long pb = plane_at(p + 3);
            const int sl = slot5(p + 3);
            issue_plane(S.old[sl], in, pb, plan);
            issue_plane(S.fr[sl], f, pb, plan);
            if constexpr (BASE)
                issue_plane(S.base[sl], B, pb, plan);
        }
        cp_async_commit();
        red_plane(p + 1);
        __syncthreads();
        // black cells of plane p over the tile; thread -> the pair (2 pr, 2 pr + 1)
        if (threadIdx.x < FT_J * (FT_K / 2)) {
            const int jj = threadIdx.x / (FT_K / 2), pr = threadIdx.x - jj * (FT_K / 2);
            const int j = j0 + jj, kp0 = k0 + 2 * pr;
            const int bodd = (p + j + kp0 + 1) & 1;  // 1: the black cell is the second of the pair
            const int kk = 2 * pr + bodd;            // tile-local k of the black cell
            const Ring r5 = ring<NSLOT>(p), r3 = ring<3>(p);
            const T *om = S.old[r5.m], *o0 = S.old[r5.z], *op = S.old[r5.p];
            const T *rm = S.rnew[r3.m], *r0 = S.rnew[r3.z], *rp = S.rnew[r3.p];
            const int cr = (jj + 1) * RK_ + (kk + 1);   // rnew coordinates of the black cell
            const int co = (jj + 2) * OROW + (kk + 4);  // old coordinates
            St<T> s;
            s.c = MG5_AT(o0, co);
            s.xp = MG5_AT(rp, cr);
            s.xm = MG5_AT(rm, cr);
            s.yp = MG5_AT(r0, cr + RK_);
            s.ym = MG5_AT(r0, cr - RK_);
            s.zp = MG5_AT(r0, cr + 1);
            s.zm = MG5_AT(r0, cr - 1);
            s.xpyp = MG5_AT(op, co + OROW);
            s.xpym = MG5_AT(op, co - OROW);
            s.xmyp = MG5_AT(om, co + OROW);
            s.xmym = MG5_AT(om, co - OROW);
            s.xpzp = MG5_AT(op, co + 1);
            s.xpzm = MG5_AT(op, co - 1);
            s.xmzp = MG5_AT(om, co + 1);
            s.xmzm = MG5_AT(om, co - 1);
            s.ypzp = MG5_AT(o0, co + OROW + 1);
            s.ypzm = MG5_AT(o0, co + OROW - 1);
            s.ymzp = MG5_AT(o0, co - OROW + 1);
            s.ymzm = MG5_AT(o0, co - OROW - 1);
            St<T> sb;
            if constexpr (BASE)
                gather_old(S.base[r5.m], S.base[r5.z], S.base[r5.p], jj + 2, kk + 4, sb);
            if (j < n && kp0 < n) {
                const long long row = ((long long)p * n + j) * n;
                const T vb = upd<T, BASE>(s, sb, S.fr[r5.z][co] + cval, cf, clamped);
                const T vr = MG5_AT(r0, (jj + 1) * RK_ + (2 * pr + 1 - bodd) + 1);
                const T v0 = bodd ? vr : vb;
                const T v1 = bodd ? vb : vr;
                if constexpr (sizeof(T) == 4) {
                    MG5_AT(reinterpret_cast<float2 *>(out + row + kp0), 0) = make_float2((float)v0, (float)v1);
                } else {
                    MG5_AT(reinterpret_cast<double2 *>(out + row + kp0), 0) = make_double2((double)v0, (double)v1);
                }
            }
        }
    }
    cp_async_wait_all();
    if (clamped)
        atomicAdd(&MG5_AT(clamp, 0), 1ull);
}

template <typename T>
cudaError_t launch_sweep_fused(const T *in, T *out, const T *f, const double *cptr, int n,
                               CoefT<T> cf, unsigned long long *clamp, cudaStream_t st, const T *B,
                               int chunk)
{
    if (!fused_ok<T>(n))
        return launch_sweep<T>(in, out, f, cptr, n, cf, clamp, st, B);
    const int tk = (n + FT_K - 1) / FT_K, tj = (n + FT_J - 1) / FT_J;
    const int tiles = tk * tj;
    int ichunk = chunk;
    if (ichunk <= 0) {
        // enough CTAs for several waves over 152 SMs, chunks of at least 8 planes
        int chunks = (8 * 152 + tiles - 1) / tiles;
        if (chunks > n / 8)
            chunks = n / 8;
        if (chunks < 1)
            chunks = 1;
        ichunk = (n + chunks - 1) / chunks;
    }
    if (ichunk > n)
        ichunk = n;
    const int chunks = (n + ichunk - 1) / ichunk;
    dim3 grid(tk, tj, chunks);
    // the shared-memory limits were raised by prepare_fused_kernels() at context creation
    if (B)
        k_sweep_fused<T, true><<<grid, FT_THREADS, sizeof(FusedSmem<T, true>), st>>>(
            in, out, f, B, cptr, n, ichunk, cf, clamp);
    else
        k_sweep_fused<T, false><<<grid, FT_THREADS, sizeof(FusedSmem<T, false>), st>>>(
            in, out, f, B, cptr, n, ichunk, cf, clamp);
    count_launch(1);
    return cudaGetLastError();
}

// set the dynamic shared-memory limits once, outside any stream capture
cudaError_t prepare_fused_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_sweep_fused<float, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(FusedSmem<float, true>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_fused<float, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(FusedSmem<float, false>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_fused<double, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(FusedSmem<double, true>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_fused<double, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(FusedSmem<double, false>));
    if (e == cudaSuccess)
        e = prepare_march_kernel();
    if (e == cudaSuccess)
        e = prepare_resid_march_kernel();
    return e;
}

template cudaError_t launch_sweep_fused<float>(const float *, float *, const float *, const double *,
                                               int, CoefT<float>, unsigned long long *, cudaStream_t,
                                               const float *, int);
template cudaError_t launch_sweep_fused<double>(const double *, double *, const double *,
                                                const double *, int, CoefT<double>,
                                                unsigned long long *, cudaStream_t, const double *, int);

}  // namespace mg5
