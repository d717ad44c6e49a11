// k_march_resid.cu -- the mixed-precision inner solve's residual of the correction
// equation, r = f + c - (op(B + e) - op(B)), restricted by 8-child means (coarse e and
// coarse r) with the residual's statistics, as a column march: one read of e, B and f and
// one write of the coarse arrays per cell.
//
// A CTA owns a 16 x 32 (j, k) tile of fine cells and marches along i over a chunk of
// planes that starts at an even plane.  Each of its 256 threads owns a pair of cells
// (j, k0 + 2 pp + {0, 1}) -- the two k-children of one coarse cell -- and computes both
// residuals on every plane.  A cell's stencil terms come from three planes of its column:
// the x-faces and the x-mixed differences from planes p +- 1 (the plane's value and its
// central differences Dy, Dz), the rest from plane p itself; each plane of a column is read
// once (rows j - 1 .. j + 1, columns k0 + 2 pp - 1 .. + 2: one 8-byte and two 4-byte shared
// loads a row), reduced to those values and kept in registers for the two planes after it.
// The rows 2J and 2J + 1 of a coarse cell are the two half-warps of one warp: after the
// odd plane the upper half passes its four children down by shuffle and the lower half
// writes the coarse cell, summing the eight children in the same order as the gather
// kernel (k_resid_restrict), so both give the same coarse values to the bit.
//
// Planes of e and B (rows j0 - 1 .. j0 + 16, 16-byte chunks k0 - 4 .. k0 + 35) and of f
// (the tile) are brought into a ring of 6 shared-memory slots by 16-byte cp.async copies,
// four planes ahead of use (a plane step of a CTA is shorter than a DRAM round trip).
//
// The grid is persistent: as many CTAs as fit on the GPU at once (one Moments partial
// each, so the final combine stays short).  The work items (chunk of planes, tile) are
// ordered chunk-major and dealt round-robin, so the CTAs running at any time hold
// neighbouring tiles at the same planes and share their halo rows in L2; the chunk length
// is chosen so that the items fill whole rounds of the grid.  Periodic in i, j, k; n a
// multiple of 32.
#include <type_traits>

#include "mg5_async.cuh"
#include "mg5_fin.cuh"

namespace mg5 {

namespace {

constexpr int RT_J = 16, RT_K = 32;            // fine tile (j, k)
constexpr int RT_THREADS = RT_J * RT_K / 2;    // one thread per cell pair
constexpr int RR = RT_J + 2;                   // e/B rows j0-1 .. j0+16
constexpr int RW = RT_K + 8;                   // e/B row: k0-4 .. k0+35
constexpr int RPL = RR * RW;                   // floats of an e or B plane
constexpr int FPL = RT_J * RT_K;               // floats of an f plane (the tile)
constexpr int RNS = 6;                         // plane slots
constexpr int RT_CH_EB = RR * (RW / 4);        // 16-byte chunks of an e (or B) plane
constexpr int RT_CH_F = RT_J * (RT_K / 4);     // ... of an f plane
constexpr int RT_CHUNKS = 2 * RT_CH_EB + RT_CH_F;
constexpr int RT_CPT = (RT_CHUNKS + RT_THREADS - 1) / RT_THREADS;

struct ResidSmem {
    float E[RNS][RPL];
    float B[RNS][RPL];
    float F[RNS][FPL];
};

template <int V>
using IC = std::integral_constant<int, V>;

// a column's plane values: the centre, face sums Y (j +- 1) and Z (k +- 1), central
// differences Dy, Dz, and the mixed difference dyz
struct PC {
    float c, Y, Z, Dy, Dz, dyz;
};

// the two columns (k = kA, kA + 1) of one plane row triple around the thread's pair;
// base points at (row j, column kA) of the plane
__device__ __forceinline__ void plane_pair(const float *base, PC &a, PC &b)
{
    float m[3], x0[3], x1[3], p2[3];   // columns kA - 1, kA, kA + 1, kA + 2 of rows j-1, j, j+1
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float *row = base + (r - 1) * RW;
        const float2 v = MG5_AT(reinterpret_cast<const float2 *>(row), 0);
        m[r] = MG5_AT(row, -1);
        x0[r] = v.x;
        x1[r] = v.y;
        p2[r] = MG5_AT(row, 2);
    }
    // column kA: k-1 = m, k = x0, k+1 = x1; column kA + 1: k-1 = x0, k = x1, k+1 = p2
    a.c = x0[1];
    a.Y = __fadd_rn(x0[2], x0[0]);
    a.Z = __fadd_rn(x1[1], m[1]);
    a.Dy = __fsub_rn(x0[2], x0[0]);
    a.Dz = __fsub_rn(x1[1], m[1]);
    a.dyz = __fsub_rn(__fsub_rn(x1[2], m[2]), __fsub_rn(x1[0], m[0]));
    b.c = x1[1];
    b.Y = __fadd_rn(x1[2], x1[0]);
    b.Z = __fadd_rn(p2[1], x0[1]);
    b.Dy = __fsub_rn(x1[2], x1[0]);
    b.Dz = __fsub_rn(p2[1], x0[1]);
    b.dyz = __fsub_rn(__fsub_rn(p2[2], x0[2]), __fsub_rn(p2[0], x0[0]));
}

// what one column keeps: plane p (all of it) and plane p - 1 (centre, Dy, Dz), for e and B
struct Col {
    PC e0, b0;                     // plane p
    float ce1, Dye1, Dze1;         // plane p - 1 of e
    float cb1, Dyb1, Dzb1;         // plane p - 1 of B
};

// residual of the column's cell on plane p, given plane p + 1 (e2, b2)
__device__ __forceinline__ float cell_resid(const Col &c, const PC &e2, const PC &b2, float fpc,
                                            const CoefT<float> &cf)
{
    const Parts2 q = parts2_from_sums(
        __fadd_rn(e2.c, c.ce1), __fadd_rn(b2.c, c.cb1), c.e0.Y, c.b0.Y, c.e0.Z, c.b0.Z,
        __fsub_rn(e2.Dy, c.Dye1), __fsub_rn(b2.Dy, c.Dyb1), __fsub_rn(e2.Dz, c.Dze1),
        __fsub_rn(b2.Dz, c.Dzb1), c.e0.dyz, c.b0.dyz);
    return __fsub_rn(fpc, cell_op_corr_parts(q, c.b0.c, c.e0.c, cf));
}

__device__ __forceinline__ void shift(Col &c, const PC &e2, const PC &b2)
{
    c.ce1 = c.e0.c;
    c.Dye1 = c.e0.Dy;
    c.Dze1 = c.e0.Dz;
    c.cb1 = c.b0.c;
    c.Dyb1 = c.b0.Dy;
    c.Dzb1 = c.b0.Dz;
    c.e0 = e2;
    c.b0 = b2;
}

__global__ void __launch_bounds__(RT_THREADS, 2)
    k_resid_restrict_march(const float *__restrict__ e, const float *__restrict__ f,
                           const float *__restrict__ Bg, const double *__restrict__ cptr, int n,
                           int ichunk, CoefT<float> cf, float *__restrict__ vc, float *__restrict__ v0c,
                           float *__restrict__ rc, Moments *__restrict__ partials, Fin fin)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    ResidSmem &S = *reinterpret_cast<ResidSmem *>(smem_raw);
    const long long n2 = (long long)n * n;
    const int nc = n >> 1;
    const float cval = (float)(MG5_AT(cptr, 0));
    const int tid = threadIdx.x;
    const int jj = tid >> 4, pp = tid & 15;        // warp w: rows 2w (lanes 0-15), 2w+1
    const int tk = n / RT_K, tiles = tk * (n / RT_J);
    const int items = tiles * ((n + ichunk - 1) / ichunk);
    MomAcc<float> acc;

    // this thread's 16-byte chunks of a plane (e, B: rows j0-1.., f: the tile)
    unsigned sdst[RT_CPT];
    const float *gp[RT_CPT];
    bool has[RT_CPT];
#pragma unroll
    for (int m = 0; m < RT_CPT; ++m) {
        const int c = tid + m * RT_THREADS;
        has[m] = c < RT_CHUNKS;
    }
    const int offE = (jj + 1) * RW + 4 + 2 * pp;   // (row j, column kA) in an e/B plane
    const int offF = jj * RT_K + 2 * pp;

    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int chunk = item / tiles, tile = item - chunk * tiles;
        const int k0 = (tile % tk) * RT_K, j0 = (tile / tk) * RT_J;
        const int i0 = chunk * ichunk;              // even
        const int i1 = min(i0 + ichunk, n);         // planes i0 .. i1 - 1 of this tile
        const int q0 = i0 - 1;                     // plane q lives in slot (q - q0) % 6
#pragma unroll
        for (int m = 0; m < RT_CPT; ++m) {
            const int c = tid + m * RT_THREADS;
            const int cm = has[m] ? c : 0;
            const float *src;
            const float *sp;
            int gj, gk;
            if (cm < 2 * RT_CH_EB) {
                const int a = cm / RT_CH_EB, w = cm - a * RT_CH_EB;
                const int r = w / (RW / 4), cc = w - r * (RW / 4);
                src = a == 0 ? e : Bg;
                sp = (a == 0 ? S.E[0] : S.B[0]) + r * RW + cc * 4;
                gj = wrap_once(j0 - 1 + r, n);
                gk = wrap_once(k0 - 4 + cc * 4, n);
            } else {
                const int w = cm - 2 * RT_CH_EB;
                const int r = w / (RT_K / 4), cc = w - r * (RT_K / 4);
                src = f;
                sp = S.F[0] + r * RT_K + cc * 4;
                gj = j0 + r;
                gk = k0 + cc * 4;
            }
            sdst[m] = (unsigned)__cvta_generic_to_shared(sp);
            gp[m] = src + (long long)wrap_once(q0, n) * n2 + (long long)gj * n + gk;
        }
        int qn = wrap_once(q0, n);
        auto issue_next = [&](int s) {
#pragma unroll
            for (int m = 0; m < RT_CPT; ++m)
                if (has[m]) {
                    const int c = tid + m * RT_THREADS;
                    const unsigned stride = c < 2 * RT_CH_EB ? RPL * 4 : FPL * 4;
                    acopy::copy16(sdst[m] + (unsigned)s * stride, gp[m]);
                }
            if (++qn == n) {
                qn = 0;
#pragma unroll
                for (int m = 0; m < RT_CPT; ++m)
                    gp[m] += n2 - (long long)n * n2;
            } else {
#pragma unroll
                for (int m = 0; m < RT_CPT; ++m)
                    gp[m] += n2;
            }
        };
        const int last = i1;   // the last plane a step reads (step i1 - 1 needs plane i1)
#pragma unroll
        for (int s = 0; s < RNS; ++s) {   // planes i0 - 1 .. i0 + 4
            if (q0 + s <= last)
                issue_next(s);
            acopy::commit();
        }
        acopy::wait<RNS - 3>();   // planes i0 - 1 .. i0 + 1
        __syncthreads();

        Col ca, cb;
        {
            PC ea, eb, ba, bb;
            plane_pair(S.E[0] + offE, ea, eb);   // plane i0 - 1
            plane_pair(S.B[0] + offE, ba, bb);
            ca.e0 = ea;
            cb.e0 = eb;
            ca.b0 = ba;
            cb.b0 = bb;
            plane_pair(S.E[1] + offE, ea, eb);   // plane i0
            plane_pair(S.B[1] + offE, ba, bb);
            shift(ca, ea, ba);
            shift(cb, eb, bb);
        }
        float v0 = 0.f, v1 = 0.f, r0 = 0.f, r1 = 0.f;   // the even plane's children of this row
        const int J = (j0 >> 1) + (jj >> 1), K = (k0 >> 1) + pp;

        // step p: plane p + 1 in slot (p - q0 + 1) % 6, f of plane p in slot (p - q0) % 6
        auto step = [&](auto SLOTc, int p) {
            constexpr int s1 = decltype(SLOTc)::value, s0 = (s1 + RNS - 1) % RNS;
            constexpr bool odd = (s1 % 2) == 1;   // p - i0 = s1 - 2 (mod 6): odd for slots 1, 3, 5
            PC ea, eb, ba, bb;
            plane_pair(S.E[s1] + offE, ea, eb);
            plane_pair(S.B[s1] + offE, ba, bb);
            const float2 fv = MG5_AT(reinterpret_cast<const float2 *>(S.F[s0] + offF), 0);
            const float ra = cell_resid(ca, ea, ba, __fadd_rn(fv.x, cval), cf);
            const float rb = cell_resid(cb, eb, bb, __fadd_rn(fv.y, cval), cf);
            acc.add(ra);
            acc.add(rb);
            const float ua = ca.e0.c, ub = cb.e0.c;
            if constexpr (!odd) {
                v0 = ua;
                v1 = ub;
                r0 = ra;
                r1 = rb;
            } else {
                // children of the coarse cell (p / 2, J, K): rows 2J (lower half-warp), 2J + 1
                const float u2 = __shfl_down_sync(0xffffffffu, v0, 16);
                const float u3 = __shfl_down_sync(0xffffffffu, v1, 16);
                const float u6 = __shfl_down_sync(0xffffffffu, ua, 16);
                const float u7 = __shfl_down_sync(0xffffffffu, ub, 16);
                const float s2 = __shfl_down_sync(0xffffffffu, r0, 16);
                const float s3 = __shfl_down_sync(0xffffffffu, r1, 16);
                const float s6 = __shfl_down_sync(0xffffffffu, ra, 16);
                const float s7 = __shfl_down_sync(0xffffffffu, rb, 16);
                if ((jj & 1) == 0) {
                    float sv = 0.f, sr = 0.f;
                    sv = __fadd_rn(sv, v0);
                    sv = __fadd_rn(sv, v1);
                    sv = __fadd_rn(sv, u2);
                    sv = __fadd_rn(sv, u3);
                    sv = __fadd_rn(sv, ua);
                    sv = __fadd_rn(sv, ub);
                    sv = __fadd_rn(sv, u6);
                    sv = __fadd_rn(sv, u7);
                    sr = __fadd_rn(sr, r0);
                    sr = __fadd_rn(sr, r1);
                    sr = __fadd_rn(sr, s2);
                    sr = __fadd_rn(sr, s3);
                    sr = __fadd_rn(sr, ra);
                    sr = __fadd_rn(sr, rb);
                    sr = __fadd_rn(sr, s6);
                    sr = __fadd_rn(sr, s7);
                    const long long t = ((long long)(p >> 1) * nc + J) * nc + K;
                    const float mv = __fmul_rn(sv, 0.125f);
                    MG5_AT(vc, t) = mv;
                    MG5_AT(v0c, t) = mv;
                    MG5_AT(rc, t) = __fmul_rn(sr, 0.125f);
                }
            }
            shift(ca, ea, ba);
            shift(cb, eb, bb);
            // bring plane p + 5 into plane p - 1's slot, then wait for plane p + 2
            if (p + 5 <= last)
                issue_next((s1 + 4) % RNS);
            acopy::commit();
            acopy::wait<RNS - 3>();
            __syncthreads();
        };
        // p - q0 + 1 = 2, 3, 4, 5, 0, 1, ... : the slot of plane p + 1 (unrolled by six)
        for (int p = i0; p < i1; p += 6) {
            step(IC<2>{}, p);
            step(IC<3>{}, p + 1);
            if (p + 2 >= i1)
                break;
            step(IC<4>{}, p + 2);
            step(IC<5>{}, p + 3);
            if (p + 4 >= i1)
                break;
            step(IC<0>{}, p + 4);
            step(IC<1>{}, p + 5);
        }
        // every copy of this tile's planes has landed before the ring is refilled
        acopy::wait<0>();
        __syncthreads();
    }
    const Moments mom = block_moments(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = mom;
    if (fin.ls)
        finalize_if_last(reinterpret_cast<double2 *>(partials), fin);
}

// CTAs of k_resid_restrict_march resident on the GPU at once (set by the preparation)
int g_resid_march_slots = 0;

}  // namespace

// raise the kernel's dynamic shared-memory limit (its static and dynamic shared memory
// together pass the 48 KiB default) and count its resident CTAs; once, outside any capture
cudaError_t prepare_resid_march_kernel()
{
    cudaError_t e = cudaFuncSetAttribute(k_resid_restrict_march,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(ResidSmem));
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess)
        e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_resid_restrict_march,
                                                          RT_THREADS, sizeof(ResidSmem));
    if (e == cudaSuccess)
        g_resid_march_slots = sms * (per_sm > 0 ? per_sm : 1);
    return e;
}

bool resid_march_ok(int n) { return n >= RT_K && n % RT_K == 0; }

cudaError_t launch_resid_restrict_march(const float *e, const float *f, const double *cptr, int n,
                                        CoefT<float> cf, float *vc, float *v0c, float *rc,
                                        double2 *partials, int *nblocks, cudaStream_t st,
                                        const float *B, const Fin &fin)
{
    if (!resid_march_ok(n) || !B)
        return cudaErrorInvalidValue;
    // one CTA per resident slot (at most kReduceBlocks: one Moments partial each)
    const int slots = g_resid_march_slots > 0 ? g_resid_march_slots : 152;
    const int g_max = slots < kReduceBlocks ? slots : kReduceBlocks;
    const int tiles = (n / RT_K) * (n / RT_J);
    // chunk length (even, at least 8 planes): the fewest plane steps per CTA, a chunk's two
    // extra planes (i0 - 1 and i1) counted, over whole rounds of g_max items
    int ichunk = n, best = -1;
    for (int c = 8; c <= n; c += 2) {
        const long long items = (long long)tiles * ((n + c - 1) / c);
        const long long rounds = (items + g_max - 1) / g_max;
        const long long cost = rounds * (c + 2);
        if (best < 0 || cost <= best) {
            best = (int)cost;
            ichunk = c;
        }
    }
    const long long items = (long long)tiles * ((n + ichunk - 1) / ichunk);
    const int g = (int)(items < g_max ? items : g_max);
    k_resid_restrict_march<<<g, RT_THREADS, sizeof(ResidSmem), st>>>(
        e, f, B, cptr, n, ichunk, cf, vc, v0c, rc, reinterpret_cast<Moments *>(partials), fin);
    *nblocks = g;
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace mg5
