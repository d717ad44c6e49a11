// k_march.cu -- the FP32 correction-form snapshot red-black sweep (the inner smoother
// of the mixed-precision solve) as a column march: one read and one write of e per
// cell per full sweep, with most of the stencil reused from registers.
//
// A CTA owns a 16 x 32 (j, k) tile and marches along i over a chunk of planes.  Each of
// its 256 tile threads owns a pair of adjacent positions (j, k0 + 2 pp + {0, 1}); at plane
// step p the pair's position with (p + 1 + j + k) even relaxes its red cell on plane p + 1
// and its black cell on plane p (red on p + 1 <=> black on p in one position), and the
// other position rests.  The snapshot semantics split the stencil cleanly:
//   * a red cell reads only old values;
//   * a black cell reads new red values at its 6 faces and old (black) values at its
//     12 edges;
// and the edge terms of a cell are differences of per-plane differences of the same
// position: with Dy_q = e(q, j+1) - e(q, j-1) and Dz_q = e(q, k+1) - e(q, k-1),
//   dxy(p) = Dy_{p+1} - Dy_{p-1},  dxz(p) = Dz_{p+1} - Dz_{p-1},
// while dyz(p), the face sums and B's parts come from the plane itself.  Each plane of a
// position is therefore read once per sweep (9 values of e, 9 of B around it), its sums
// and differences stay in registers for the two steps that use them, and the new red
// values of the black cells' in-plane faces pass through shared memory; a black cell's
// x-faces are the thread's own red values of the planes above and below.
//
// The black cells at the tile's edge need the new red values of the ring of positions
// around the tile; 50 more threads own pairs of ring positions and compute their red
// cells the same way (red only).  Threads past the tile also bring the planes of e, B
// and f into a ring of 6 shared-memory slots with bulk asynchronous copies
// (cp.async.bulk, one per row segment, completion counted on one mbarrier per slot),
// three plane steps ahead of use.  320 threads and 62 KB of shared memory a CTA: two
// CTAs per SM, so one CTA's barrier waits overlap the other's work.
//
// Every cell is updated by the same arithmetic on the same operands, in the same order,
// as the gather-based kernels (cell_update_corr_parts), so the result is the same sweep
// to the bit.  Periodic in i, j, k; n a multiple of 32; out of place.
#include "mg5_kernels.cuh"

namespace mg5 {

namespace {

constexpr int MT_J = 16, MT_K = 32;           // tile (j, k)
constexpr int MT_TILE = MT_J * MT_K / 2;      // tile threads: one per column pair
constexpr int MT_RINGP = (MT_K + 2) + MT_J;   // ring threads: pairs of ring positions (50)
constexpr int MT_THREADS = 320;               // 256 tile + 50 ring + 14 that only copy
constexpr int MR = MT_J + 4;                  // plane rows j0-2 .. j0+17
constexpr int MO = MT_K + 8;                  // plane row: k0-4 .. k0+35 (16-byte aligned)
constexpr int MPL = MR * MO;                  // floats of one plane
constexpr int MNS = 6;                        // plane slots
constexpr int RNR = MT_J + 2, RNO = MT_K + 2; // new red values: j0-1 .. j0+16, k0-1 .. k0+32
constexpr int RNP = RNR * RNO;
constexpr int MT_COPIERS = 3 * MR;            // one thread per copied row (60)
constexpr unsigned MT_PLANE_BYTES = 3u * MR * MO * 4u;           // e, B, f rows of a plane
constexpr long long kWaitLimit = 1ll << 26;   // mbarrier polls before giving up
static_assert(MT_TILE + MT_RINGP <= MT_THREADS && MT_COPIERS <= MT_THREADS - MT_TILE, "roles");

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

// values a position keeps between its two active steps (plane p: read two steps earlier as
// plane p + 2; plane p - 1: read two steps earlier as plane p + 1)
struct ColCache {
    float cE0, DyE0, DzE0, dyzE0, cB0, DyB0, DzB0, dyzB0, YB0, ZB0;   // plane p
    float DyEm, DzEm, DyBm, DzBm, cBm, rm;                            // plane p - 1, red(p - 1)
};

// 3 x 3 neighbourhood of a position on one plane, reduced to what the cell arithmetic uses
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

// A thread's two positions (adjacent cells, so of opposite colours): plane offsets, offsets
// in the new-red array, and for tile threads the output offset within a plane.
struct Pos {
    int off, rn;
};

__global__ void __launch_bounds__(MT_THREADS, 2)
    k_sweep_march(const float *__restrict__ in, float *__restrict__ out, const float *__restrict__ f,
                  const float *__restrict__ Bg, const double *__restrict__ cptr, int n, int ichunk,
                  CoefT<float> cf, unsigned long long *clamp)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MarchSmem &S = *reinterpret_cast<MarchSmem *>(smem_raw);
    const int k0 = blockIdx.x * MT_K, j0 = blockIdx.y * MT_J;
    const int i0 = blockIdx.z * ichunk;
    const int i1 = min(i0 + ichunk, n);
    const int q0 = i0 - 2;        // first plane brought in; plane q lives in slot (q - q0) % MNS
    const int last = i1 + 1;      // the last plane any step reads
    const float cval = (float)(*cptr);
    const long long n2 = (long long)n * n;
    const int tid = threadIdx.x;
    const bool tile = tid < MT_TILE;
    const bool ring = !tile && tid < MT_TILE + MT_RINGP;
    const int ct = tid - MT_TILE;   // copier index (threads past the tile)
    bool clamped = false, fault = false;

    if (tid == 0) {
        for (int s = 0; s < MNS; ++s)
            mbar_init(&S.bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // copier threads: row `ct` of e, B or f of plane q into slot s
    const float *csrc = nullptr;
    float *cdst0 = nullptr;
    long long crow = 0;
    if (ct >= 0 && ct < MT_COPIERS) {
        const int a = ct / MR, jr = ct - a * MR;
        csrc = a == 0 ? in : (a == 1 ? Bg : f);
        cdst0 = (a == 0 ? S.E[0] : (a == 1 ? S.B[0] : S.F[0])) + jr * MO;
        crow = (long long)wrapn(j0 - 2 + jr, n) * n;
    }
    const bool kwrap = !(k0 > 0 && k0 + MT_K < n);
    const int kl = k0 > 0 ? k0 - 4 : n - 4, kr = k0 + MT_K < n ? k0 + MT_K : 0;
    auto issue_plane = [&](int q, int s) {
        if (ct == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&S.bar[s], MT_PLANE_BYTES);
        }
        if (csrc) {
            const float *row = csrc + (long long)wrapn(q, n) * n2 + crow;
            float *dst = cdst0 + s * MPL;
            if (!kwrap) {
                bulk_g2s(dst, row + k0 - 4, MO * 4, &S.bar[s]);
            } else {
                bulk_g2s(dst, row + kl, 16, &S.bar[s]);
                bulk_g2s(dst + 4, row + k0, MT_K * 4, &S.bar[s]);
                bulk_g2s(dst + 4 + MT_K, row + kr, 16, &S.bar[s]);
            }
        }
    };
    auto wait_slot = [&](int s, unsigned par) {
        long long it = 0;
        while (!mbar_try_wait(&S.bar[s], par)) {
            if (++it > kWaitLimit) {   // never expected: record it and go on
                fault = true;
                break;
            }
        }
    };
    if (ct >= 0)
        for (int q = q0; q < q0 + MNS && q <= last; ++q)
            issue_plane(q, q - q0);

    // the thread's two positions (j, k global; A and B adjacent)
    int jA, kA, jB, kB;
    if (tile) {
        jA = jB = j0 + (tid >> 4);
        kA = k0 + 2 * (tid & 15);
        kB = kA + 1;
    } else if (ring) {
        const int r = tid - MT_TILE;
        if (r < MT_K + 2) {   // top and bottom rows: pairs along k
            const int m = r < (MT_K + 2) / 2 ? r : r - (MT_K + 2) / 2;
            jA = jB = r < (MT_K + 2) / 2 ? j0 - 1 : j0 + MT_J;
            kA = k0 - 1 + 2 * m;
            kB = kA + 1;
        } else {              // left and right columns: pairs along j
            const int r2 = r - (MT_K + 2);
            const int m = r2 < MT_J / 2 ? r2 : r2 - MT_J / 2;
            kA = kB = r2 < MT_J / 2 ? k0 - 1 : k0 + MT_K;
            jA = j0 + 2 * m;
            jB = jA + 1;
        }
    } else {
        jA = jB = j0;
        kA = k0;
        kB = k0 + 1;
    }
    const Pos pA{(jA - j0 + 2) * MO + (kA - k0 + 4), (jA - j0 + 1) * RNO + (kA - k0 + 1)};
    const Pos pB{(jB - j0 + 2) * MO + (kB - k0 + 4), (jB - j0 + 1) * RNO + (kB - k0 + 1)};
    // step p relaxes the position with (p + 1 + j + k) even: A on steps of one parity
    const bool a_even = ((q0 + 1 + jA + kA) & 1) == 0;   // A active on steps q0, q0 + 2, ...
    const Pos p0 = a_even ? pA : pB, p1 = a_even ? pB : pA;
    const bool first0 = a_even ? (kA < kB || jA < jB) : (kB < kA || jB < jA);
    float *orow = out + (long long)(tile ? jA : j0) * n + (tile ? kA : k0);
    ColCache c0{}, c1{};
    float rprev = 0.0f;   // red value of the step before (its plane's red cell)

    // One step p with slots s0 (plane p), s1 (p + 1), s2 (p + 2) and the active position's
    // cache.  warm: a step before the chunk (no black cell, no output; plane p's values are
    // read here instead of two steps earlier).
    auto step = [&](int p, int s0, int s1, int s2, const Pos &ps, bool pfirst, ColCache &cc,
                    bool warm) {
        if (tile || ring) {
            const int off = ps.off;
            if (warm) {
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
            // red cell (p + 1) of the position: old values throughout
            const Parts2 qr = parts_from(pk_add(pr2(e2.c, b2.c), pr2(cc.cE0, cc.cB0)),
                                         pr2(e1.Y, b1.Y), pr2(e1.Z, b1.Z),
                                         pk_sub(pr2(e2.Dy, b2.Dy), pr2(cc.DyE0, cc.DyB0)),
                                         pk_sub(pr2(e2.Dz, b2.Dz), pr2(cc.DzE0, cc.DzB0)),
                                         pr2(e1.dyz, b1.dyz));
            const float r1 = cell_update_corr_parts(qr, b1.c, e1.c, S.F[s1][off] + cval, cf, clamped);
            S.RN[(p + 1) & 1][ps.rn] = r1;
            if (tile && !warm) {
                // black cell (p) of the position: new red faces, old edges
                const float *rn = S.RN[p & 1] + ps.rn;
                const float sye = rn[RNO] + rn[-RNO], sze = rn[1] + rn[-1];
                const Parts2 qb = parts_from(pk_add(pr2(r1, b1.c), pr2(cc.rm, cc.cBm)),
                                             pr2(sye, cc.YB0), pr2(sze, cc.ZB0),
                                             pk_sub(pr2(e1.Dy, b1.Dy), pr2(cc.DyEm, cc.DyBm)),
                                             pk_sub(pr2(e1.Dz, b1.Dz), pr2(cc.DzEm, cc.DzBm)),
                                             pr2(cc.dyzE0, cc.dyzB0));
                const float b0v = cell_update_corr_parts(qb, cc.cB0, cc.cE0, S.F[s0][off] + cval,
                                                         cf, clamped);
                float2 v;
                v.x = pfirst ? b0v : rprev;
                v.y = pfirst ? rprev : b0v;
                *reinterpret_cast<float2 *>(orow + (long long)p * n2) = v;
            }
            // keep plane p + 2 as the position's plane p, plane p + 1 as its plane p - 1
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
        }
    };

    // slots and mbarrier phases of planes p, p + 1, p + 2, kept incrementally
    int s0 = 0, s1 = 1, s2 = 2;
    unsigned ph2 = 0;   // phase parity of slot s2's current plane
    auto advance = [&]() {
        s0 = s1;
        s1 = s2;
        s2 = s2 == MNS - 1 ? 0 : s2 + 1;
        if (s2 == 0)
            ph2 ^= 1u;
    };
    // warm-up: steps q0 and q0 + 1 compute the red cells of planes i0 - 1 and i0
    wait_slot(0, 0);
    wait_slot(1, 0);
    wait_slot(2, 0);
    step(q0, s0, s1, s2, p0, first0, c0, true);
    __syncthreads();
    advance();
    wait_slot(s2, ph2);
    step(q0 + 1, s0, s1, s2, p1, !first0, c1, true);
    __syncthreads();
    // plane p - 1's slot is free after step p: plane p + 5 goes there (3 steps before use)
    if (ct >= 0 && q0 + 6 <= last)
        issue_plane(q0 + 6, 0);
    int p = i0;
    for (; p < i1; ++p) {
        advance();
        wait_slot(s2, ph2);
        if (((p - i0) & 1) == 0)
            step(p, s0, s1, s2, p0, first0, c0, false);
        else
            step(p, s0, s1, s2, p1, !first0, c1, false);
        __syncthreads();
        if (ct >= 0 && p + 5 <= last)
            issue_plane(p + 5, s0 == 0 ? MNS - 1 : s0 - 1);
    }
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
        // about six waves of two CTAs per SM over 152 SMs, chunks of at least 16 planes
        int chunks = (6 * 2 * 152 + tiles - 1) / tiles;
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
