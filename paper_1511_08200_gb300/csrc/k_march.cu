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
// cells the same way (red only).  All 320 threads bring the planes of e, B and f into a
// ring of 6 shared-memory slots with 16-byte cp.async copies (two a thread a plane),
// three plane steps ahead of use; each thread waits for its own copies before the step's
// barrier.  320 threads and 67 KB of shared memory a CTA: two CTAs per SM, so one CTA's
// barrier waits overlap the other's work.
//
// The plane values, sums and differences of e and B travel as (e, B) pairs through the
// packed FP32 instructions (two lanes an instruction).  Every cell is updated by the same
// arithmetic on the same operands, in the same order, as the gather-based kernels
// (parts2_of, cell_update_corr_parts), so the result is the same sweep to the bit.  Periodic in i, j, k; n a multiple of 32; out of place.
#include <type_traits>

#include "mg5_async.cuh"
#include "mg5_kernels.cuh"

namespace mg5 {

namespace {

constexpr int MT_J = 16, MT_K = 32;           // tile (j, k)
constexpr int MT_TILE = MT_J * MT_K / 2;      // tile threads: one per position pair
constexpr int MT_RINGP = (MT_K + 2) + MT_J;   // ring threads: pairs of ring positions (50)
constexpr int MT_THREADS = 320;               // 256 tile + 50 ring + 14 that only copy
constexpr int MR = MT_J + 4;                  // plane rows j0-2 .. j0+17
constexpr int MW = MT_K + 8;                  // copied row: k0-4 .. k0+35 (16-byte chunks)
constexpr int MO = MW + 4;                    // row stride: 4 floats of padding, so that the
                                              // ring's column cells (rows 2 apart) spread over
                                              // 4 banks instead of 2
constexpr int MPL = MR * MO;                  // floats of one plane
constexpr int MNS = 6;                        // plane slots
constexpr int RNR = MT_J + 2, RNO = MT_K + 2; // new red values: j0-1 .. j0+16, k0-1 .. k0+32
constexpr int RNP = RNR * RNO;
constexpr int MT_CHUNKS = 3 * MR * (MW / 4);  // 16-byte chunks of one plane of e, B and f
constexpr int MT_CPT = (MT_CHUNKS + MT_THREADS - 1) / MT_THREADS;   // chunks a thread copies
static_assert(MT_TILE + MT_RINGP <= MT_THREADS, "roles");

struct MarchSmem {
    float P[3][MNS][MPL];   // e (old values), B, f: plane slots
    float RN[2][RNP];       // new red values of planes p and p + 1
};


// values a position keeps between its two active steps, (e, B) pairs where both are used
// (plane p: read two steps earlier as plane p + 2; plane p - 1: read two steps earlier as
// plane p + 1)
struct ColCache {
    float2 c0, Dy0, Dz0, dyz0;   // plane p
    float YB0, ZB0;              // plane p, B only (the black cell's e faces are new red values)
    float2 Dym, Dzm;             // plane p - 1
    float2 rBm;                  // plane p - 1: (the red value, B's centre)
};

// 3 x 3 neighbourhood of a position on one plane as (e, B) pairs, reduced to what the cell
// arithmetic uses; the packed FP32 instructions do e and B together
struct PlaneCol2 {
    float2 c, Y, Z, Dy, Dz, dyz;
};

__device__ __forceinline__ PlaneCol2 plane_col2(const float *be, const float *bb)
{
    const auto ld = [&](int o) { return make_float2(MG5_AT(be, o), MG5_AT(bb, o)); };
    PlaneCol2 r;
    r.c = ld(0);
    const float2 yp = ld(MO), ym = ld(-MO), zp = ld(1), zm = ld(-1);
    const float2 pp = ld(MO + 1), pm = ld(MO - 1), mp = ld(-MO + 1), mm = ld(-MO - 1);
    r.Y = pk_add(yp, ym);
    r.Z = pk_add(zp, zm);
    r.Dy = pk_sub(yp, ym);
    r.Dz = pk_sub(zp, zm);
    r.dyz = pk_sub(pk_sub(pp, pm), pk_sub(mp, mm));
    return r;
}

// A thread's position: its plane offset and its offset in the new-red array.
struct Pos {
    int off, rn;
};

template <int V>
using IC = std::integral_constant<int, V>;

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
    const int q0 = i0 - 2;        // first plane brought in; plane q lives in slot (q - q0) % 6
    const int last = i1 + 1;      // the last plane any step reads
    const float cval = (float)(MG5_AT(cptr, 0));
    const long long n2 = (long long)n * n;
    const int tid = threadIdx.x;
    const bool tile = tid < MT_TILE;
    const bool ring = !tile && tid < MT_TILE + MT_RINGP;
    bool clamped = false;

    // This thread's 16-byte chunks of a plane: the shared address in slot 0 and a global
    // pointer into the next plane to bring in (advanced one plane per copy, wrapped at n).
    unsigned sdst[MT_CPT];
    const float *gp[MT_CPT];
    bool has[MT_CPT];
#pragma unroll
    for (int m = 0; m < MT_CPT; ++m) {
        const int c = tid + m * MT_THREADS;
        has[m] = c < MT_CHUNKS;
        const int cm = has[m] ? c : 0;
        const int a = cm / (MR * (MW / 4)), w = cm - a * (MR * (MW / 4));
        const int r = w / (MW / 4), cc = w - r * (MW / 4);
        const float *src = a == 0 ? in : (a == 1 ? Bg : f);
        sdst[m] = (unsigned)__cvta_generic_to_shared(&S.P[a][0][r * MO + cc * 4]);
        gp[m] = src + (long long)wrap_once(q0, n) * n2 + (long long)wrap_once(j0 - 2 + r, n) * n +
                wrap_once(k0 - 4 + cc * 4, n);
    }
    int qn = wrap_once(q0, n);   // wrapped index of the next plane to bring in
    auto issue_next = [&](int s) {
#pragma unroll
        for (int m = 0; m < MT_CPT; ++m)
            if (has[m])
                acopy::copy16(sdst[m] + (unsigned)(s * MPL * 4), gp[m]);
        if (++qn == n) {
            qn = 0;
#pragma unroll
            for (int m = 0; m < MT_CPT; ++m)
                gp[m] += n2 - (long long)n * n2;
        } else {
#pragma unroll
            for (int m = 0; m < MT_CPT; ++m)
                gp[m] += n2;
        }
    };
    // planes q0 .. q0 + 4 now; every step then brings in plane p + 5 (three steps ahead)
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        if (q0 + s <= last)
            issue_next(s);
        acopy::commit();
    }

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
    const Pos pos[2] = {a_even ? pA : pB, a_even ? pB : pA};
    const bool first[2] = {a_even, !a_even};   // tile pairs: A is the pair's first cell
    float *optr = out + (long long)i0 * n2 + (long long)(tile ? jA : j0) * n + (tile ? kA : k0);
    ColCache cc[2] = {};
    float rprev = 0.0f;   // red value of the step before (its plane's red cell)
    const float *E = S.P[0][0], *Bs = S.P[1][0], *F = S.P[2][0];

    // One step p: planes p, p + 1, p + 2 in slots S0, S0 + 1, S0 + 2 (mod 6), position set
    // SET.  warm: a step before the chunk (no black cell, no output; plane p's values are
    // read here instead of two steps earlier).
    auto step = [&](auto S0c, auto SETc, bool warm) {
        constexpr int s0 = decltype(S0c)::value, set = decltype(SETc)::value;
        constexpr int s1 = (s0 + 1) % MNS, s2 = (s0 + 2) % MNS;
        if (tile || ring) {
            ColCache &c = cc[set];
            const Pos ps = pos[set];
            const float *E0 = E + s0 * MPL + ps.off, *E1 = E + s1 * MPL + ps.off,
                        *E2 = E + s2 * MPL + ps.off;
            const float *B0 = Bs + s0 * MPL + ps.off, *B1 = Bs + s1 * MPL + ps.off,
                        *B2 = Bs + s2 * MPL + ps.off;
            if (warm) {
                const PlaneCol2 q0 = plane_col2(E0, B0);
                c.c0 = q0.c;
                c.Dy0 = q0.Dy;
                c.Dz0 = q0.Dz;
                c.dyz0 = q0.dyz;
                c.YB0 = q0.Y.y;
                c.ZB0 = q0.Z.y;
            }
            const PlaneCol2 q2 = plane_col2(E2, B2), q1 = plane_col2(E1, B1);
            // red cell (p + 1) of the position: old values throughout (x faces: p + 2, p)
            const Parts2 qr = parts2_from_pairs(pk_add(q2.c, c.c0), q1.Y, q1.Z, pk_sub(q2.Dy, c.Dy0),
                                                pk_sub(q2.Dz, c.Dz0), q1.dyz);
            const float r1 = cell_update_corr_parts(qr, q1.c.y, q1.c.x, MG5_AT(F, s1 * MPL + ps.off) + cval,
                                                    cf, clamped);
            MG5_AT(S.RN[(set + 1) & 1], ps.rn) = r1;   // plane p + 1 (p - i0 has the parity of set)
            const float2 rB1 = make_float2(r1, q1.c.y);
            if (tile && !warm) {
                // black cell (p) of the position: new red faces, old edges
                const float *rn = S.RN[set & 1] + ps.rn;
                const float sye = __fadd_rn(MG5_AT(rn, RNO), MG5_AT(rn, -RNO)), sze = __fadd_rn(MG5_AT(rn, 1), MG5_AT(rn, -1));
                const Parts2 qb = parts2_from_pairs(
                    pk_add(rB1, c.rBm), make_float2(sye, c.YB0),
                    make_float2(sze, c.ZB0), pk_sub(q1.Dy, c.Dym), pk_sub(q1.Dz, c.Dzm), c.dyz0);
                const float b0v = cell_update_corr_parts(qb, c.c0.y, c.c0.x,
                                                         MG5_AT(F, s0 * MPL + ps.off) + cval, cf, clamped);
                float2 v;
                v.x = first[set] ? b0v : rprev;
                v.y = first[set] ? rprev : b0v;
                MG5_AT(reinterpret_cast<float2 *>(optr), 0) = v;
            }
            // keep plane p + 2 as the position's plane p, plane p + 1 as its plane p - 1
            c.c0 = q2.c;
            c.Dy0 = q2.Dy;
            c.Dz0 = q2.Dz;
            c.dyz0 = q2.dyz;
            c.YB0 = q2.Y.y;
            c.ZB0 = q2.Z.y;
            c.Dym = q1.Dy;
            c.Dzm = q1.Dz;
            c.rBm = rB1;
            rprev = r1;
        }
    };
    // after step p: bring in plane p + 5 (into plane p - 1's slot, free during step p), then
    // wait until at most two copy groups are pending: the plane the next step reads last has
    // landed (this thread's chunks; the barrier makes every thread's chunks visible)
    auto finish = [&](auto S0c, int p) {
        constexpr int s0 = decltype(S0c)::value;
        if (p + 5 <= last)
            issue_next((s0 + 5) % MNS);
        acopy::commit();
        acopy::wait<2>();
        __syncthreads();
    };
    acopy::wait<2>();   // planes q0 .. q0 + 2
    __syncthreads();
    // warm-up: the red cells of planes i0 - 1 and i0
    step(IC<0>{}, IC<0>{}, true);
    finish(IC<0>{}, q0);
    step(IC<1>{}, IC<1>{}, true);
    finish(IC<1>{}, q0 + 1);
    // plane p's slot is (p - q0) % 6: steps i0, i0 + 1, ... use slots 2, 3, 4, 5, 0, 1 and
    // position sets 0, 1, 0, 1, 0, 1 (unrolled by twelve: every slot offset is a constant)
    for (int p = i0; p < i1;) {
        step(IC<2>{}, IC<0>{}, false);
        finish(IC<2>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<3>{}, IC<1>{}, false);
        finish(IC<3>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<4>{}, IC<0>{}, false);
        finish(IC<4>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<5>{}, IC<1>{}, false);
        finish(IC<5>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<0>{}, IC<0>{}, false);
        finish(IC<0>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<1>{}, IC<1>{}, false);
        finish(IC<1>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        // the same six again: each position set's cached values are replaced an even number
        // of times a loop pass, so they can alternate between two register sets
        step(IC<2>{}, IC<0>{}, false);
        finish(IC<2>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<3>{}, IC<1>{}, false);
        finish(IC<3>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<4>{}, IC<0>{}, false);
        finish(IC<4>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<5>{}, IC<1>{}, false);
        finish(IC<5>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<0>{}, IC<0>{}, false);
        finish(IC<0>{}, p);
        optr += n2;
        if (++p >= i1)
            break;
        step(IC<1>{}, IC<1>{}, false);
        finish(IC<1>{}, p);
        optr += n2;
        ++p;
    }
    if (clamped)
        atomicAdd(&MG5_AT(clamp, 0), 1ull);
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
