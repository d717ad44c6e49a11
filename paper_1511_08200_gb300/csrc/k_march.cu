// k_march.cu -- the FP32 correction-form snapshot red-black sweep (the inner smoother
// of the mixed-precision solve) as a column march: one read and one write of e per
// cell per full sweep, with most of the stencil reused from registers.
//
// A CTA owns a 32 x 32 (j, k) tile and marches along i over a chunk of planes.  Its
// 512 tile threads each own a pair of columns (j, k0 + 2 pp + {0, 1}); at plane step p
// the pair's column c with (p + 1 + j + c) even relaxes its red cell on plane p + 1 and
// its black cell on plane p (in the same column: red on p + 1 <=> black on p), and the
// other column rests.  The snapshot semantics split the stencil cleanly:
//   * a red cell reads only old values;
//   * a black cell reads new red values at its 6 faces and old (black) values at its
//     12 edges;
// and the edge terms of a cell are differences of per-plane differences of the same
// column: with Dy_q = e(q, j+1) - e(q, j-1) and Dz_q = e(q, k+1) - e(q, k-1),
//   dxy(p) = Dy_{p+1} - Dy_{p-1},  dxz(p) = Dz_{p+1} - Dz_{p-1},
// and dyz(p), the face sums and B's parts come from the plane itself.  Each plane of a
// column is therefore read once per sweep (9 values of e, 9 of B, around the column),
// its differences are kept in registers for the two steps that need them, and the new
// red values of the black cells' in-plane faces come through shared memory.  The
// black cells' x-faces are the thread's own red values of the planes above and below.
//
// The new red values on the ring around the tile (the black cells at the tile's edge
// need them) are computed by three extra warps from full gathers; the same warps bring
// the planes of e, B and f into a ring of 6 shared-memory slots with bulk asynchronous
// copies (cp.async.bulk, one per row segment, completion counted on an mbarrier per
// slot), 3 plane steps ahead of use.
//
// Every cell is updated by the same arithmetic on the same operands, in the same order,
// as the gather-based kernels (cell_update_corr_parts), so the result is the same sweep
// to the bit.  Periodic in i, j, k; n a multiple of 32; out of place.
#include "mg5_kernels.cuh"

namespace mg5 {

namespace {

constexpr int MT_J = 32, MT_K = 32;           // tile (j, k)
constexpr int MT_TILE = MT_J * MT_K / 2;      // tile threads: one per column pair
constexpr int MT_RING = 96;                   // ring warps: ring red cells and copies
constexpr int MT_THREADS = MT_TILE + MT_RING;
constexpr int MR = MT_J + 4;                  // plane rows j0-2 .. j0+33
constexpr int MO = MT_K + 8;                  // plane row: k0-4 .. k0+35 (16-byte aligned)
constexpr int MPL = MR * MO;                  // floats of one plane
constexpr int MNS = 6;                        // plane slots
constexpr int RNR = MT_J + 2, RNO = MT_K + 2; // new red values: j0-1 .. j0+32, k0-1 .. k0+32
constexpr int RNP = RNR * RNO;
constexpr int MT_RINGCELLS = 2 * (MT_K + 2) / 2 + 2 * MT_J / 2;   // 66 red cells per plane
constexpr unsigned MT_PLANE_BYTES = 3u * MR * MO * 4u;           // e, B, f rows of a plane
constexpr long long kWaitLimit = 1ll << 26;   // mbarrier polls before giving up

struct MarchSmem {
    float E[MNS][MPL];
    float B[MNS][MPL];
    float F[MNS][MPL];
    float RN[2][RNP];
    unsigned long long bar[MNS];
};

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
        " selp.u32 %0, 1, 0, P;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// global -> shared bulk copy of `bytes` (multiple of 16, both ends 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ int wrapn(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// values a column keeps between its two active steps (plane p: read two steps earlier as
// plane p + 2; plane p - 1: read two steps earlier as plane p + 1)
struct ColCache {
    float cE0, DyE0, DzE0, dyzE0, cB0, DyB0, DzB0, dyzB0, YB0, ZB0;   // plane p
    float DyEm, DzEm, DyBm, DzBm, cBm, rm;                            // plane p - 1, red(p - 1)
};

// 3 x 3 neighbourhood of a column on one plane, reduced to what the cell arithmetic uses
struct PlaneCol {
    float c, Y, Z, Dy, Dz, dyz;
};

__device__ __forceinline__ PlaneCol plane_col(const float *base)
{
    PlaneCol r;
    r.c = base[0];
    const float yp = base[MO], ym = base[-MO], zp = base[1], zm = base[-1];
    const float pp = base[MO + 1], pm = base[MO - 1], mp = base[-MO + 1], mm = base[-MO - 1];
    r.Y = yp + ym;
    r.Z = zp + zm;
    r.Dy = yp - ym;
    r.Dz = zp - zm;
    r.dyz = (pp - pm) - (mp - mm);
    return r;
}

__device__ __forceinline__ float2 pr2(float x, float y) { return make_float2(x, y); }

// (e, B) parts of a cell from its face sums and its mixed differences
__device__ __forceinline__ Parts2 parts_from(float2 sx, float2 sy, float2 sz, float2 dxy,
                                             float2 dxz, float2 dyz)
{
    Parts2 q;
    q.S = pk_add(pk_add(sx, sy), sz);
    q.a = pk_sub(sx, sy);
    q.b = pk_sub(sx, sz);
    q.c = pk_sub(sy, sz);
    q.dxy = dxy;
    q.dxz = dxz;
    q.dyz = dyz;
    return q;
}

__global__ void __launch_bounds__(MT_THREADS, 1)
    k_sweep_march(const float *__restrict__ in, float *__restrict__ out, const float *__restrict__ f,
                  const float *__restrict__ Bg, const double *__restrict__ cptr, int n, int ichunk,
                  CoefT<float> cf, unsigned long long *clamp)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MarchSmem &S = *reinterpret_cast<MarchSmem *>(smem_raw);
    const int k0 = blockIdx.x * MT_K, j0 = blockIdx.y * MT_J;
    const int i0 = blockIdx.z * ichunk;
    const int i1 = min(i0 + ichunk, n);
    const int q0 = i0 - 2;   // first plane brought in; plane q lives in slot (q - q0) % MNS
    const float cval = (float)(*cptr);
    const long long n2 = (long long)n * n;
    const int tid = threadIdx.x;
    const bool tile = tid < MT_TILE;
    const int rt = tid - MT_TILE;   // ring thread index (tile threads: negative)
    bool clamped = false, fault = false;

    if (tid == 0) {
        for (int s = 0; s < MNS; ++s)
            mbar_init(&S.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ring threads: bring plane q (its rows of e, B, f) into its slot
    auto issue_plane = [&](int q) {
        const int s = (q - q0) % MNS;
        if (rt == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&S.bar[s], MT_PLANE_BYTES);
        }
        const long long pb = (long long)wrapn(q, n) * n2;
        for (int idx = rt; idx < 3 * MR; idx += MT_RING) {
            const int a = idx / MR, jr = idx - a * MR;
            const float *src = a == 0 ? in : (a == 1 ? Bg : f);
            float *dst = (a == 0 ? S.E[s] : (a == 1 ? S.B[s] : S.F[s])) + jr * MO;
            const float *row = src + pb + (long long)wrapn(j0 - 2 + jr, n) * n;
            if (k0 > 0 && k0 + MT_K < n) {
                bulk_g2s(dst, row + k0 - 4, MO * 4, &S.bar[s]);
            } else {
                bulk_g2s(dst, row + (k0 > 0 ? k0 - 4 : n - 4), 16, &S.bar[s]);
                bulk_g2s(dst + 4, row + k0, MT_K * 4, &S.bar[s]);
                bulk_g2s(dst + 4 + MT_K, row + (k0 + MT_K < n ? k0 + MT_K : 0), 16, &S.bar[s]);
            }
        }
    };
    // every thread: wait until plane q has landed
    auto wait_plane = [&](int q) {
        const int u = q - q0;
        unsigned long long *bar = &S.bar[u % MNS];
        const unsigned par = (unsigned)((u / MNS) & 1);
        long long it = 0;
        while (!mbar_try_wait(bar, par)) {
            if (++it > kWaitLimit) {   // never expected: record it and go on
                fault = true;
                break;
            }
        }
    };
    auto slot = [&](int q) { return (q - q0) % MNS; };

    const int last_plane = i1 + 1;   // the last plane any step reads
    if (!tile)
        for (int q = q0; q < q0 + MNS && q <= last_plane; ++q)
            issue_plane(q);

    // tile thread geometry
    const int jj = tile ? tid >> 4 : 0;   // row in the tile
    const int pp = tid & 15;              // column pair
    const int rowE = (jj + 2) * MO;       // plane offset of the thread's row
    ColCache ca{}, cb{};                  // column sets of even / odd steps from i0
    float rprev = 0.0f;                   // red value of the step before (plane p's red cell)

    // One step p.  warm: a step before the chunk (no black cell, no output; plane p's
    // column values are read here instead of two steps earlier).
    auto step = [&](int p, ColCache &cc, bool warm) {
        wait_plane(p + 2);
        if (warm && p == q0)
            for (int q = q0; q < q0 + 2; ++q)
                wait_plane(q);
        if (tile) {
            const int j = j0 + jj;
            const int cl = 2 * pp + ((p + 1 + j) & 1);   // local k of the active column
            const int off = rowE + cl + 4;
            const int s0 = slot(p), s1 = slot(p + 1), s2 = slot(p + 2);
            if (warm) {   // plane p of the column, normally kept from two steps earlier
                const PlaneCol e0 = plane_col(S.E[s0] + off), b0 = plane_col(S.B[s0] + off);
                cc.cE0 = e0.c;
                cc.DyE0 = e0.Dy;
                cc.DzE0 = e0.Dz;
                cc.dyzE0 = e0.dyz;
                cc.cB0 = b0.c;
                cc.DyB0 = b0.Dy;
                cc.DzB0 = b0.Dz;
                cc.dyzB0 = b0.dyz;
                cc.YB0 = b0.Y;
                cc.ZB0 = b0.Z;
            }
            const PlaneCol e2 = plane_col(S.E[s2] + off), b2 = plane_col(S.B[s2] + off);
            const PlaneCol e1 = plane_col(S.E[s1] + off), b1 = plane_col(S.B[s1] + off);
            // red cell (p + 1, j, c): old values throughout
            const Parts2 qr = parts_from(pk_add(pr2(e2.c, b2.c), pr2(cc.cE0, cc.cB0)),
                                         pr2(e1.Y, b1.Y), pr2(e1.Z, b1.Z),
                                         pk_sub(pr2(e2.Dy, b2.Dy), pr2(cc.DyE0, cc.DyB0)),
                                         pk_sub(pr2(e2.Dz, b2.Dz), pr2(cc.DzE0, cc.DzB0)),
                                         pr2(e1.dyz, b1.dyz));
            const float r1 = cell_update_corr_parts(qr, b1.c, e1.c, S.F[s1][off] + cval, cf, clamped);
            S.RN[(p + 1) & 1][(jj + 1) * RNO + cl + 1] = r1;
            if (!warm) {
                // black cell (p, j, c): new red faces, old edges
                const float *rn = S.RN[p & 1] + (jj + 1) * RNO + cl + 1;
                const float sye = rn[RNO] + rn[-RNO], sze = rn[1] + rn[-1];
                const Parts2 qb = parts_from(pk_add(pr2(r1, b1.c), pr2(cc.rm, cc.cBm)),
                                             pr2(sye, cc.YB0), pr2(sze, cc.ZB0),
                                             pk_sub(pr2(e1.Dy, b1.Dy), pr2(cc.DyEm, cc.DyBm)),
                                             pk_sub(pr2(e1.Dz, b1.Dz), pr2(cc.DzEm, cc.DzBm)),
                                             pr2(cc.dyzE0, cc.dyzB0));
                const float b0v = cell_update_corr_parts(qb, cc.cB0, cc.cE0, S.F[s0][off] + cval,
                                                         cf, clamped);
                const bool bfirst = (cl & 1) == 0;   // the black cell is the pair's first
                float2 v;
                v.x = bfirst ? b0v : rprev;
                v.y = bfirst ? rprev : b0v;
                *reinterpret_cast<float2 *>(out + (long long)p * n2 + (long long)j * n + k0 + 2 * pp) = v;
            }
            // keep plane p + 2 as the column's plane p, plane p + 1 as its plane p - 1
            cc.cE0 = e2.c;
            cc.DyE0 = e2.Dy;
            cc.DzE0 = e2.Dz;
            cc.dyzE0 = e2.dyz;
            cc.cB0 = b2.c;
            cc.DyB0 = b2.Dy;
            cc.DzB0 = b2.Dz;
            cc.dyzB0 = b2.dyz;
            cc.YB0 = b2.Y;
            cc.ZB0 = b2.Z;
            cc.DyEm = e1.Dy;
            cc.DzEm = e1.Dz;
            cc.DyBm = b1.Dy;
            cc.DzBm = b1.Dz;
            cc.cBm = b1.c;
            cc.rm = r1;
            rprev = r1;
        } else if (rt < MT_RINGCELLS && !(warm && p == q0)) {
            // red cell of plane p + 1 on the ring around the tile, from a full gather
            const int P = p + 1;
            int j, k;
            if (rt < 34) {
                const int m = rt < 17 ? rt : rt - 17;
                j = rt < 17 ? j0 - 1 : j0 + MT_J;
                k = k0 - 1 + ((P + j + k0 - 1) & 1) + 2 * m;
            } else {
                const int m = rt < 50 ? rt - 34 : rt - 50;
                k = rt < 50 ? k0 - 1 : k0 + MT_K;
                j = j0 + ((P + k + j0) & 1) + 2 * m;
            }
            const int jr = j - j0 + 2, kc = k - k0 + 4;
            const int o = jr * MO + kc;
            const float *em = S.E[slot(p)], *e0 = S.E[slot(P)], *ep = S.E[slot(P + 1)];
            const float *bm = S.B[slot(p)], *b0 = S.B[slot(P)], *bp = S.B[slot(P + 1)];
            St<float> se, sb;
            auto g = [&](const float *xm, const float *x0, const float *xp, St<float> &t) {
                t.c = x0[o];
                t.xp = xp[o];
                t.xm = xm[o];
                t.yp = x0[o + MO];
                t.ym = x0[o - MO];
                t.zp = x0[o + 1];
                t.zm = x0[o - 1];
                t.xpyp = xp[o + MO];
                t.xpym = xp[o - MO];
                t.xmyp = xm[o + MO];
                t.xmym = xm[o - MO];
                t.xpzp = xp[o + 1];
                t.xpzm = xp[o - 1];
                t.xmzp = xm[o + 1];
                t.xmzm = xm[o - 1];
                t.ypzp = x0[o + MO + 1];
                t.ypzm = x0[o + MO - 1];
                t.ymzp = x0[o - MO + 1];
                t.ymzm = x0[o - MO - 1];
            };
            g(em, e0, ep, se);
            g(bm, b0, bp, sb);
            const float v = cell_update_corr(se, sb, S.F[slot(P)][o] + cval, cf, clamped);
            S.RN[P & 1][(j - j0 + 1) * RNO + (k - k0 + 1)] = v;
        }
        __syncthreads();
        // plane p - 1's slot is free now: bring in plane p + 5 (3 steps before its use)
        if (!tile && p + 5 <= last_plane && p - 1 >= q0)
            issue_plane(p + 5);
    };

    // warm-up: red of planes i0 - 1 and i0 (tile columns), ring red of plane i0
    step(i0 - 2, ca, true);
    step(i0 - 1, cb, true);
    int p = i0;
    for (; p + 1 < i1; p += 2) {
        step(p, ca, false);
        step(p + 1, cb, false);
    }
    if (p < i1)
        step(p, ca, false);
    if (clamped)
        atomicAdd(clamp, 1ull);
    if (fault)
        atomicOr(clamp, kSweepFaultBit);
}

}  // namespace

bool march_ok(int n) { return n >= MT_K && n % MT_K == 0 && n % MT_J == 0; }

cudaError_t launch_sweep_march(const float *in, float *out, const float *f, const float *B,
                               const double *cptr, int n, CoefT<float> cf,
                               unsigned long long *clamp, cudaStream_t st, int chunk)
{
    if (!march_ok(n) || !B)
        return cudaErrorInvalidValue;
    const int tiles = (n / MT_K) * (n / MT_J);
    int ichunk = chunk;
    if (ichunk <= 0) {
        // about three waves of one CTA per SM, chunks of at least 16 planes
        int chunks = (3 * 152 + tiles - 1) / tiles;
        if (chunks > n / 16)
            chunks = n / 16;
        if (chunks < 1)
            chunks = 1;
        ichunk = (n + chunks - 1) / chunks;
    }
    if (ichunk > n)
        ichunk = n;
    const int chunks = (n + ichunk - 1) / ichunk;
    dim3 grid(n / MT_K, n / MT_J, chunks);
    k_sweep_march<<<grid, MT_THREADS, sizeof(MarchSmem), st>>>(in, out, f, B, cptr, n, ichunk, cf,
                                                              clamp);
    count_launch(1);
    return cudaGetLastError();
}

cudaError_t prepare_march_kernel()
{
    return cudaFuncSetAttribute(k_sweep_march, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(MarchSmem));
}

}  // namespace mg5
