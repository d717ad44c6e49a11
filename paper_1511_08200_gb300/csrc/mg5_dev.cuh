// mg5_dev.cuh -- device helpers shared by the mg5 kernels: the 19-point
// stencil gather, the cell arithmetic of Eq. (eomvarphi) and deterministic
// block reductions.
//
// The discrete operator: D_aa = (phi[+a] + phi[-a] - 2 phi)/h^2,
// D_ab = (phi[+a+b] - phi[+a-b] - phi[-a+b] + phi[-a-b])/(4 h^2), L = sum D_aa.
// (lap)^2 - (d_i d_j phi)^2 = (2/3) L^2 - Sigma with
// Sigma = (1/3) sum_{a<b} (D_aa - D_bb)^2 + 2 sum_{a<b} D_ab^2, which does not
// depend on the centre value (the centre cancels in D_aa - D_bb and is not
// used by D_ab).  So with every neighbour fixed, the cell's equation
// L + alpha((2/3) L^2 - Sigma) = rhs is a quadratic in L whose physical root
// (continuous with alpha -> 0) is L = 2 b / (1 + sqrt(1 + 8 alpha b / 3)),
// b = rhs + alpha Sigma, and phi_ijk = (sum of faces - h^2 L) / 6.
// That value is the fixed point of the Newton update of Eq. (newton).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "mg5_bounds.cuh"

namespace mg5 {

// Per-grid constants of the cell arithmetic.
template <typename T>
struct CoefT {
    T h2;      // h^2
    T inv_h2;  // 1/h^2
    T a_h4;    // alpha / h^4
    T k8;      // 8 alpha / 3
    T k23;     // 2 alpha / 3
    T s23;     // (2/3) alpha / h^4: weight of t = a^2 + b c in alpha Sigma
    T s8;      // alpha / (8 h^4): weight of d2 = sum (4 h^2 D_ab)^2 in alpha Sigma
    float k8f;   // 8 alpha / 3, for the FP32 estimate of the FP64 root
    float k43f;  // 4 alpha / 3 (slope of the quadratic is 1 + k43 L)
    T s3;        // alpha / (3 h^4): weight of the (a, b, c) terms of alpha Sigma(., .)
    T k43h;      // (4 alpha / 3) / h^2: beta' = 1 + k43h (S_B - 6 B_c)
    T inv2k23;   // 1 / (2 k23) (0 when alpha = 0, where it is never used)
    T om1;       // omega - 1: a smoothing update is v + omega (v_root - v)
    int relaxed;   // om1 != 0, as an integer: the FP64 sweeps test it per cell, and an FP64
                   // compare would run on the FP64 pipe
    T k23i4;     // (2 alpha / 3) / h^4: op = Lh (1/h^2 + k23i4 Lh) - ..., Lh = h^2 L
    T w6;        // omega / 6: ... = (omega / 6) (S - h^2 L) + (1 - omega) v
    T omc;       // 1 - omega
};

template <typename T>
__host__ __device__ inline CoefT<T> make_coef(double h, double alpha, double omega = 1.0)
{
    CoefT<T> c;
    const double h4 = h * h * h * h;
    c.h2 = (T)(h * h);
    c.inv_h2 = (T)(1.0 / (h * h));
    c.a_h4 = (T)(alpha / h4);
    c.k8 = (T)(8.0 * alpha / 3.0);
    c.k23 = (T)(2.0 * alpha / 3.0);
    c.s23 = (T)(2.0 * alpha / (3.0 * h4));
    c.s8 = (T)(alpha / (8.0 * h4));
    c.k8f = (float)(8.0 * alpha / 3.0);
    c.k43f = (float)(4.0 * alpha / 3.0);
    c.s3 = (T)(alpha / (3.0 * h4));
    c.k43h = (T)(4.0 * alpha / (3.0 * h * h));
    c.inv2k23 = (T)(alpha > 0.0 ? 3.0 / (4.0 * alpha) : 0.0);
    c.om1 = (T)(omega - 1.0);
    c.relaxed = omega != 1.0;
    c.k23i4 = (T)(2.0 * alpha / (3.0 * h4));
    c.w6 = (T)(omega / 6.0);
    c.omc = (T)(1.0 - omega);
    return c;
}

// The 19 values the cell arithmetic reads: centre, 6 faces, 12 edges.
template <typename T>
struct St {
    T c, xp, xm, yp, ym, zp, zm;
    T xpyp, xpym, xmyp, xmym;
    T xpzp, xpzm, xmzp, xmzm;
    T ypzp, ypzm, ymzp, ymzm;
};

// Row offsets of the 9 (i', j') rows around (i, j); k offsets are added by the gather.
struct Rows {
    long long r00, rp0, rm0, r0p, r0m, rpp, rpm, rmp, rmm;
};

__device__ __forceinline__ Rows periodic_rows(int n, int i, int j)
{
    const int ip = (i == n - 1) ? 0 : i + 1, im = (i == 0) ? n - 1 : i - 1;
    const int jp = (j == n - 1) ? 0 : j + 1, jm = (j == 0) ? n - 1 : j - 1;
    const long long N = n;
    Rows r;
    r.r00 = ((long long)i * N + j) * N;
    r.rp0 = ((long long)ip * N + j) * N;
    r.rm0 = ((long long)im * N + j) * N;
    r.r0p = ((long long)i * N + jp) * N;
    r.r0m = ((long long)i * N + jm) * N;
    r.rpp = ((long long)ip * N + jp) * N;
    r.rpm = ((long long)ip * N + jm) * N;
    r.rmp = ((long long)im * N + jp) * N;
    r.rmm = ((long long)im * N + jm) * N;
    return r;
}

// Box of dims (d0, d1, d2) without wrapping; (i, j) must have both neighbours.
__device__ __forceinline__ Rows box_rows(int d1, int d2, int i, int j)
{
    const long long D1 = d1, D2 = d2;
    Rows r;
    r.r00 = ((long long)i * D1 + j) * D2;
    r.rp0 = ((long long)(i + 1) * D1 + j) * D2;
    r.rm0 = ((long long)(i - 1) * D1 + j) * D2;
    r.r0p = ((long long)i * D1 + j + 1) * D2;
    r.r0m = ((long long)i * D1 + j - 1) * D2;
    r.rpp = ((long long)(i + 1) * D1 + j + 1) * D2;
    r.rpm = ((long long)(i + 1) * D1 + j - 1) * D2;
    r.rmp = ((long long)(i - 1) * D1 + j + 1) * D2;
    r.rmm = ((long long)(i - 1) * D1 + j - 1) * D2;
    return r;
}

// Faces from F, edges from E, the centre from C.
template <typename T>
__device__ __forceinline__ void gather3(const T *F, const T *E, const T *C, const Rows &r, int k,
                                        int kp, int km, St<T> &s)
{
    s.c = MG5_AT(C, r.r00 + k);
    s.xp = MG5_AT(F, r.rp0 + k);
    s.xm = MG5_AT(F, r.rm0 + k);
    s.yp = MG5_AT(F, r.r0p + k);
    s.ym = MG5_AT(F, r.r0m + k);
    s.zp = MG5_AT(F, r.r00 + kp);
    s.zm = MG5_AT(F, r.r00 + km);
    s.xpyp = MG5_AT(E, r.rpp + k);
    s.xpym = MG5_AT(E, r.rpm + k);
    s.xmyp = MG5_AT(E, r.rmp + k);
    s.xmym = MG5_AT(E, r.rmm + k);
    s.xpzp = MG5_AT(E, r.rp0 + kp);
    s.xpzm = MG5_AT(E, r.rp0 + km);
    s.xmzp = MG5_AT(E, r.rm0 + kp);
    s.xmzm = MG5_AT(E, r.rm0 + km);
    s.ypzp = MG5_AT(E, r.r0p + kp);
    s.ypzm = MG5_AT(E, r.r0p + km);
    s.ymzp = MG5_AT(E, r.r0m + kp);
    s.ymzm = MG5_AT(E, r.r0m + km);
}

// Faces (and the centre) from F, edges from E.
template <typename T>
__device__ __forceinline__ void gather(const T *F, const T *E, const Rows &r, int k, int kp,
                                       int km, St<T> &s)
{
    gather3(F, E, F, r, k, kp, km, s);
}

// The 19 offsets of a cell's stencil within one array (St order), for kernels that
// visit the same cell many times (the single-CTA coarsest-grid solves) and compute
// them once instead of on every visit.
struct Nbr {
    int o[19];
};

__device__ __forceinline__ Nbr nbr_of(const Rows &r, int k, int kp, int km)
{
    Nbr b;
    const int r00 = (int)r.r00, rp0 = (int)r.rp0, rm0 = (int)r.rm0, r0p = (int)r.r0p,
              r0m = (int)r.r0m;
    b.o[0] = r00 + k;
    b.o[1] = rp0 + k;
    b.o[2] = rm0 + k;
    b.o[3] = r0p + k;
    b.o[4] = r0m + k;
    b.o[5] = r00 + kp;
    b.o[6] = r00 + km;
    b.o[7] = (int)r.rpp + k;
    b.o[8] = (int)r.rpm + k;
    b.o[9] = (int)r.rmp + k;
    b.o[10] = (int)r.rmm + k;
    b.o[11] = rp0 + kp;
    b.o[12] = rp0 + km;
    b.o[13] = rm0 + kp;
    b.o[14] = rm0 + km;
    b.o[15] = r0p + kp;
    b.o[16] = r0p + km;
    b.o[17] = r0m + kp;
    b.o[18] = r0m + km;
    return b;
}

template <typename T>
__device__ __forceinline__ void gather_nbr(const T *a, const Nbr &b, St<T> &s)
{
    s.c = MG5_AT(a, b.o[0]);
    s.xp = MG5_AT(a, b.o[1]);
    s.xm = MG5_AT(a, b.o[2]);
    s.yp = MG5_AT(a, b.o[3]);
    s.ym = MG5_AT(a, b.o[4]);
    s.zp = MG5_AT(a, b.o[5]);
    s.zm = MG5_AT(a, b.o[6]);
    s.xpyp = MG5_AT(a, b.o[7]);
    s.xpym = MG5_AT(a, b.o[8]);
    s.xmyp = MG5_AT(a, b.o[9]);
    s.xmym = MG5_AT(a, b.o[10]);
    s.xpzp = MG5_AT(a, b.o[11]);
    s.xpzm = MG5_AT(a, b.o[12]);
    s.xmzp = MG5_AT(a, b.o[13]);
    s.xmzm = MG5_AT(a, b.o[14]);
    s.ypzp = MG5_AT(a, b.o[15]);
    s.ypzm = MG5_AT(a, b.o[16]);
    s.ymzp = MG5_AT(a, b.o[17]);
    s.ymzm = MG5_AT(a, b.o[18]);
}

// S = sum of the 6 faces; t and d2 with Sigma h^4 = (2/3) t + d2 / 8:
// a = sx - sy, b = sx - sz, c = sy - sz (sx = faces along x, ...) satisfy c = b - a,
// so (1/3)(a^2 + b^2 + c^2) = (2/3)(a^2 + b c) = (2/3) t; d2 = dxy^2 + dxz^2 + dyz^2
// with dab = 4 h^2 D_ab.  Every term is a difference of neighbours: no cancellation
// against the (much larger) field values.
template <typename T>
__device__ __forceinline__ void stencil_parts(const St<T> &s, T &S, T &t, T &d2)
{
    const T sx = s.xp + s.xm, sy = s.yp + s.ym, sz = s.zp + s.zm;
    S = sx + sy + sz;
    const T a = sx - sy, b = sx - sz, c = sy - sz;
    t = a * a + b * c;
    const T dxy = (s.xpyp - s.xpym) - (s.xmyp - s.xmym);
    const T dxz = (s.xpzp - s.xpzm) - (s.xmzp - s.xmzm);
    const T dyz = (s.ypzp - s.ypzm) - (s.ymzp - s.ymzm);
    d2 = dxy * dxy + dxz * dxz + dyz * dyz;
}

// Physical root of (2 alpha/3) L^2 + L - b = 0, L = 2b / (1 + sqrt(1 + 8 alpha b / 3));
// a negative discriminant is clamped to zero (L = 2b) and flagged.
//
// FP32: the closed form with the fast approximate square root and divide (the
// FP32 inner solve of the mixed mode needs ~1e-6, not correct rounding).
// FP64: GB300 executes FP64 at 1/64 of the FP32 rate, and the IEEE square root
// and divide sequences would be ~40% of the cell's FP64 instructions.  The root
// is instead estimated in FP32 and refined by one Newton step of the quadratic
// q(L) = (2 alpha/3) L^2 + L - b (the update of Eq. newton) in FP64, with the
// FP32 reciprocal of q'(L) held fixed.  With e the estimate's error (~3e-7 of L)
// the step leaves |1 - q'(L) r| e + (2 alpha/3) e^2 / q', q' = sqrt(disc): about
// 3e-7 (6e-8 + 1.5e-7 |q' - 1| / q') of L, 2e-14 for q' near 1 and at most 1e-13 for
// q' >= 0.5; a cell's update then moves phi by that fraction of h^2 L / 6, far below
// the solves' tolerances.  The branch test runs in FP32 (the FP32 discriminant is
// within ~1e-7 of the FP64 one): below df = 0.25 (q' < 0.5: strongly nonlinear cells,
// near the double root, or clamped) the closed form runs in FP64 instead.
__device__ __forceinline__ float physical_root(float b, float k8, bool &clamped)
{
    float disc = fmaf(k8, b, 1.0f);
    if (disc <= 0.0f) {
        clamped = clamped || disc < 0.0f;
        return 2.0f * b;
    }
    return __fdividef(2.0f * b, 1.0f + disc * rsqrtf(disc));
}

__device__ __forceinline__ float physical_root(float b, const CoefT<float> &cf, bool &clamped)
{
    return physical_root(b, cf.k8, clamped);
}

// ---- FP64 <-> FP32 conversions on the integer pipes ---------------------------
// GB300 executes the F2F conversions between FP64 and FP32 on the FP64 pipe at the FP64
// rate, so in the FP64-bound kernels (the FP64 smoother, the mixed mode's FP64 residual)
// each conversion costs as much as an FP64 add.  These give the same values from the bit
// patterns with a few integer instructions, for every input in FP32's normal range (and
// zero, infinities and NaN); FP32 subnormals are flushed to zero (values below 1.2e-38,
// which the fields and residuals here do not reach).
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned ed = (hi >> 20) & 0x7ffu;
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);   // the 23 kept fraction bits
    const unsigned rest = lo & 0x1fffffffu;                     // the 29 dropped ones
    // round to nearest, ties to even; a carry out of the fraction steps the exponent
    // (up to infinity), as rounding does
    const unsigned up = (rest > 0x10000000u) | ((rest == 0x10000000u) & m);
    unsigned bits = (((ed - 896u) << 23) | m) + up;
    bits = ed <= 896u ? 0u : bits;
    bits = ed >= 1151u ? ((ed == 2047u && (m | rest) != 0u) ? 0x7fc00000u : 0x7f800000u) : bits;
    return __uint_as_float((hi & 0x80000000u) | bits);
}

__device__ __forceinline__ double f32_to_f64(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    unsigned hi = ((u & 0x7fffffffu) >> 3) + (896u << 20);   // exponent + 1023 - 127
    hi = e == 0u ? 0u : hi;
    hi = e == 255u ? hi + (896u << 20) : hi;                  // infinity, NaN: exponent 2047
    const unsigned lo = e == 0u ? 0u : (u << 29);
    return __hiloint2double((int)((u & 0x80000000u) | hi), (int)lo);
}

__device__ __forceinline__ double physical_root(double b, const CoefT<double> &cf, bool &clamped)
{
#ifdef MG5_IEEE_ROOT
    double disc = 1.0 + cf.k8 * b;
    if (disc < 0.0) {
        disc = 0.0;
        clamped = true;
    }
    return 2.0 * b / (1.0 + sqrt(disc));
#else
    const float bf = f64_to_f32_rn(b);
    const float df = fmaf(cf.k8f, bf, 1.0f);
    if (df < 0.25f) {
        const double disc = fma(cf.k8, b, 1.0);
        if (disc < 0.0) {
            clamped = true;
            return 2.0 * b;
        }
        return 2.0 * b / (1.0 + sqrt(disc));
    }
    const float Lf = __fdividef(2.0f * bf, 1.0f + sqrtf(df));
    const double r = f32_to_f64(__frcp_rn(fmaf(cf.k43f, Lf, 1.0f)));
    const double L = f32_to_f64(Lf);
    return fma(-fma(fma(cf.k23, L, 1.0), L, -b), r, L);
#endif
}

// New centre value solving the cell's equation with op(...) = rhs.
template <typename T>
__device__ __forceinline__ T cell_update(const St<T> &s, T rhs, const CoefT<T> &cf, bool &clamped)
{
    T S, t, d2;
    stencil_parts(s, S, t, d2);
    const T b = rhs + cf.s8 * d2 + cf.s23 * t;   // rhs + alpha Sigma
    const T L = physical_root(b, cf, clamped);
    const T r6 = S - cf.h2 * L;   // 6 v_root
    return cf.relaxed ? cf.w6 * r6 + cf.omc * s.c : r6 * (T)(1.0 / 6.0);
}

// op(phi) at the cell = L + alpha((2/3) L^2 - Sigma).
template <typename T>
__device__ __forceinline__ T cell_op(const St<T> &s, const CoefT<T> &cf)
{
    T S, t, d2;
    stencil_parts(s, S, t, d2);
    const T L = (S - (T)6 * s.c) * cf.inv_h2;
    return L + cf.k23 * L * L - cf.s8 * d2 - cf.s23 * t;
}

// fc - op(phi) at the cell (fc = f + c), op in units of Lh = h^2 L = S - 6 v:
// op = Lh (1/h^2 + k23i4 Lh) - s8 d2 - s23 t, so that after the stencil parts the residual
// is one FP64 add and five fused multiply-adds (cell_op then a subtraction take eight).
template <typename T>
__device__ __forceinline__ T cell_residual(const St<T> &s, T fc, const CoefT<T> &cf)
{
    T S, t, d2;
    stencil_parts(s, S, t, d2);
    const T Lh = fma((T)-6, s.c, S);
    const T u = fma(cf.k23i4, Lh, cf.inv_h2);
    const T r = fma(cf.s8, d2, fma(-Lh, u, fc));
    return fma(cf.s23, t, r);
}

// ---- correction form (mixed precision) -------------------------------------
// With a fixed base B and a correction e, op(B + e) - op(B) expands without
// cancellation against op(B):
//   L_e + alpha [ (4/3) L_B L_e + (2/3) L_e^2 - 2 Sigma(B, e) - Sigma(e) ],
// Sigma(., .) the symmetric bilinear form of Sigma.  Sigma(B, e) and
// Sigma(e) do not depend on e_ijk, so the cell equation is again a quadratic
// in L_e:  (2 alpha/3) L_e^2 + beta' L_e - b' = 0, beta' = 1 + (4 alpha/3) L_B,
// b' = rhs + alpha (2 Sigma(B, e) + Sigma(e)), physical root (the one that
// makes L_B + L_e the physical root of the full equation)
// L_e = (sqrt(D) - beta') / (4 alpha / 3) = 2 b' / (beta' + sqrt(D)),
// D = beta'^2 + 8 alpha b' / 3; the second form for beta' >= 0, the first otherwise.
template <typename T>
struct Parts {
    T S, a, b, c, dxy, dxz, dyz;  // S = faces; a,b,c = sx-sy, sx-sz, sy-sz
};

template <typename T>
__device__ __forceinline__ Parts<T> parts_of(const St<T> &s)
{
    Parts<T> p;
    const T sx = s.xp + s.xm, sy = s.yp + s.ym, sz = s.zp + s.zm;
    p.S = sx + sy + sz;
    p.a = sx - sy;
    p.b = sx - sz;
    p.c = sy - sz;
    p.dxy = (s.xpyp - s.xpym) - (s.xmyp - s.xmym);
    p.dxz = (s.xpzp - s.xpzm) - (s.xmzp - s.xmzm);
    p.dyz = (s.ypzp - s.ypzm) - (s.ymzp - s.ymzm);
    return p;
}

// Sigma(p, q) * h^4
template <typename T>
__device__ __forceinline__ T sig_bil(const Parts<T> &p, const Parts<T> &q)
{
    return (p.a * q.a + p.b * q.b + p.c * q.c) * (T)(1.0 / 3.0) +
           (p.dxy * q.dxy + p.dxz * q.dxz + p.dyz * q.dyz) * (T)0.125;
}

template <typename T>
__device__ __forceinline__ T cell_update_corr(const St<T> &e, const St<T> &B, T rhs,
                                              const CoefT<T> &cf, bool &clamped)
{
    const Parts<T> pe = parts_of(e), pb = parts_of(B);
    const T LB = (pb.S - (T)6 * B.c) * cf.inv_h2;
    const T bp = (T)1 + (T)2 * cf.k23 * LB;
    const T b = rhs + cf.a_h4 * ((T)2 * sig_bil(pb, pe) + sig_bil(pe, pe));
    T disc = bp * bp + cf.k8 * b;
    if (disc < (T)0) {
        disc = (T)0;
        clamped = true;
    }
    // the same root in the form without cancellation for either sign of beta'
    // (beta' < 0 needs alpha > 0, so k23 > 0 there)
    const T sq = sqrt(disc);
    const T L = bp >= (T)0 ? (T)2 * b / (bp + sq) : (sq - bp) / ((T)2 * cf.k23);
    const T r6 = pe.S - cf.h2 * L;
    return cf.relaxed ? cf.w6 * r6 + cf.omc * e.c : r6 * (T)(1.0 / 6.0);
}

// FP32 correction form, the inner sweep of the mixed mode.  The same update as the
// template above, arranged for issue rate: the parts of e and of B are computed as
// pairs by the packed FP32 instructions (two lanes per instruction on sm_100 and
// later); 2 Sigma(B, e) + Sigma(e) = sum_t w_t e_t (2 B_t + e_t) as one sum with
// its weights folded into the per-grid constants; the root with the fast square
// root and divide (the inner solve needs ~1e-6, the FP64 outer loop corrects it).
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(d)
        : "l"(*reinterpret_cast<const unsigned long long *>(&a)),
          "l"(*reinterpret_cast<const unsigned long long *>(&b)));
    return *reinterpret_cast<const float2 *>(&d);
}

// Parts of e and B as (e, B) pairs, and the merged form
// X = sum_{a,b,c} e_t (2 B_t + e_t), Y = sum_{dxy,dxz,dyz} e_t (2 B_t + e_t).
struct Parts2 {
    float2 S, a, b, c, dxy, dxz, dyz;
};

__device__ __forceinline__ Parts2 parts2_of(const St<float> &e, const St<float> &B)
{
    const auto pr = [](float x, float y) { return make_float2(x, y); };   // (e, B)
    Parts2 q;
    const float2 sx = pk_add(pr(e.xp, B.xp), pr(e.xm, B.xm));
    const float2 sy = pk_add(pr(e.yp, B.yp), pr(e.ym, B.ym));
    const float2 sz = pk_add(pr(e.zp, B.zp), pr(e.zm, B.zm));
    q.S = pk_add(pk_add(sx, sy), sz);
    q.a = pk_sub(sx, sy);
    q.b = pk_sub(sx, sz);
    q.c = pk_sub(sy, sz);
    q.dxy = pk_sub(pk_sub(pr(e.xpyp, B.xpyp), pr(e.xpym, B.xpym)),
                   pk_sub(pr(e.xmyp, B.xmyp), pr(e.xmym, B.xmym)));
    q.dxz = pk_sub(pk_sub(pr(e.xpzp, B.xpzp), pr(e.xpzm, B.xpzm)),
                   pk_sub(pr(e.xmzp, B.xmzp), pr(e.xmzm, B.xmzm)));
    q.dyz = pk_sub(pk_sub(pr(e.ypzp, B.ypzp), pr(e.ypzm, B.ypzm)),
                   pk_sub(pr(e.ymzp, B.ymzp), pr(e.ymzm, B.ymzm)));
    return q;
}

// alpha (2 Sigma(B, e) + Sigma(e)), the weights folded into s3 = alpha / (3 h^4), s8 = alpha / (8 h^4)
// Every operation of the update is written as an explicitly rounded intrinsic, so the compiler
// cannot contract it differently in different kernels: every kernel that calls it (gather,
// fused, column march) computes the same sweep to the bit.
__device__ __forceinline__ float sigma_corr(const Parts2 &q, const CoefT<float> &cf)
{
    // sum_t e_t (2 B_t + e_t) as a chain of multiply-adds
    const auto u = [](float2 v) { return __fmaf_rn(2.0f, v.y, v.x); };
    const float X = __fmaf_rn(q.a.x, u(q.a), __fmaf_rn(q.b.x, u(q.b), __fmul_rn(q.c.x, u(q.c))));
    const float Y =
        __fmaf_rn(q.dxy.x, u(q.dxy), __fmaf_rn(q.dxz.x, u(q.dxz), __fmul_rn(q.dyz.x, u(q.dyz))));
    return __fmaf_rn(cf.s3, X, __fmul_rn(cf.s8, Y));
}

// (e, B) parts of a cell from its face sums sx, sy, sz and mixed differences, each half in
// scalar arithmetic: the same roundings as the packed pairs of parts2_of (kernels that build
// the sums from separately cached e and B plane values use this).
__device__ __forceinline__ Parts2 parts2_from_sums(float sxe, float sxb, float sye, float syb,
                                                   float sze, float szb, float dxye, float dxyb,
                                                   float dxze, float dxzb, float dyze, float dyzb)
{
    Parts2 q;
    q.S = make_float2(__fadd_rn(__fadd_rn(sxe, sye), sze), __fadd_rn(__fadd_rn(sxb, syb), szb));
    q.a = make_float2(__fsub_rn(sxe, sye), __fsub_rn(sxb, syb));
    q.b = make_float2(__fsub_rn(sxe, sze), __fsub_rn(sxb, szb));
    q.c = make_float2(__fsub_rn(sye, sze), __fsub_rn(syb, szb));
    q.dxy = make_float2(dxye, dxyb);
    q.dxz = make_float2(dxze, dxzb);
    q.dyz = make_float2(dyze, dyzb);
    return q;
}

// (e, B) parts of a cell from its packed face sums sx, sy, sz and mixed differences: the
// packed operations of parts2_of in the same order (kernels that build the sums from cached
// plane values, two lanes an instruction).
__device__ __forceinline__ Parts2 parts2_from_pairs(float2 sx, float2 sy, float2 sz, float2 dxy,
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

// The update from the (e, B) parts, B's centre Bc and e's centre ec (used by omega != 1).
__device__ __forceinline__ float cell_update_corr_parts(const Parts2 &q, float Bc, float ec, float rhs,
                                                        const CoefT<float> &cf, bool &clamped)
{
    const float bp = __fmaf_rn(cf.k43h, __fmaf_rn(-6.0f, Bc, q.S.y), 1.0f);   // beta' = 1 + (4 alpha/3) L_B
    const float bq = __fadd_rn(rhs, sigma_corr(q, cf));                        // b'
    float disc = __fmaf_rn(bp, bp, __fmul_rn(cf.k8, bq));
    clamped = clamped || disc < 0.0f;
    disc = fmaxf(disc, 0.0f);
    // both root forms evaluated and one selected: no branch
    const float sq = disc > 0.0f ? __fmul_rn(disc, rsqrtf(disc)) : 0.0f;
    const float Lp = __fdividef(__fmul_rn(2.0f, bq), __fadd_rn(bp, sq));
    const float Lm = __fmul_rn(__fsub_rn(sq, bp), cf.inv2k23);
    const float L = bp >= 0.0f ? Lp : Lm;
    const float r6 = __fmaf_rn(-cf.h2, L, q.S.x);
    // (omega / 6) r6 + (1 - omega) e_c; for omega = 1 it is r6 / 6 rounded once
    return __fmaf_rn(cf.w6, r6, __fmul_rn(cf.omc, ec));
}

__device__ __forceinline__ float cell_update_corr(const St<float> &e, const St<float> &B, float rhs,
                                                  const CoefT<float> &cf, bool &clamped)
{
    return cell_update_corr_parts(parts2_of(e, B), B.c, e.c, rhs, cf, clamped);
}

// op(B + e) - op(B) in FP32: L_e + (2 alpha / 3) L_e (2 L_B + L_e) - alpha (2 Sigma(B, e) + Sigma(e)),
// from the (e, B) parts and the centres (explicitly rounded: every residual kernel agrees)
__device__ __forceinline__ float cell_op_corr_parts(const Parts2 &q, float Bc, float ec,
                                                    const CoefT<float> &cf)
{
    const float LB = __fmul_rn(__fmaf_rn(-6.0f, Bc, q.S.y), cf.inv_h2);
    const float Le = __fmul_rn(__fmaf_rn(-6.0f, ec, q.S.x), cf.inv_h2);
    return __fsub_rn(__fmaf_rn(__fmul_rn(cf.k23, Le), __fmaf_rn(2.0f, LB, Le), Le),
                     sigma_corr(q, cf));
}

__device__ __forceinline__ float cell_op_corr(const St<float> &e, const St<float> &B,
                                              const CoefT<float> &cf)
{
    return cell_op_corr_parts(parts2_of(e, B), B.c, e.c, cf);
}

template <typename T>
__device__ __forceinline__ T cell_op_corr(const St<T> &e, const St<T> &B, const CoefT<T> &cf)
{
    const Parts<T> pe = parts_of(e), pb = parts_of(B);
    const T LB = (pb.S - (T)6 * B.c) * cf.inv_h2;
    const T Le = (pe.S - (T)6 * e.c) * cf.inv_h2;
    return Le + cf.k23 * Le * ((T)2 * LB + Le) -
           cf.a_h4 * ((T)2 * sig_bil(pb, pe) + sig_bil(pe, pe));
}

// Dispatch on the presence of a base field.
template <typename T, bool BASE>
__device__ __forceinline__ T upd(const St<T> &s, const St<T> &B, T rhs, const CoefT<T> &cf,
                                 bool &clamped)
{
    if constexpr (BASE)
        return cell_update_corr(s, B, rhs, cf, clamped);
    else
        return cell_update(s, rhs, cf, clamped);
}

template <typename T, bool BASE>
__device__ __forceinline__ T opr(const St<T> &s, const St<T> &B, const CoefT<T> &cf)
{
    if constexpr (BASE)
        return cell_op_corr(s, B, cf);
    else
        return cell_op(s, cf);
}

// fc - opr: the residual of a cell with right-hand side fc
template <typename T, bool BASE>
__device__ __forceinline__ T resid_of(const St<T> &s, const St<T> &B, T fc, const CoefT<T> &cf)
{
    if constexpr (BASE)
        return fc - cell_op_corr(s, B, cf);
    else
        return cell_residual(s, fc, cf);
}

// ---- residual statistics -----------------------------------------------------
// The stopping test needs ||r - mean r||; forming it as sum r^2 - N mean^2 cancels when
// |mean| is far above the spread of r (a stale compatibility constant, a warm start, a
// source with a non-zero mean).  A set of values is therefore kept as shifted sums: the
// count n, a shift K that is one of the values, S = sum (x - K) and Q = sum (x - K)^2;
// then mean = K + S / n and M2 = sum (x - mean)^2 = Q - S^2 / n, and since K lies
// within the data, S / n is of the order of the spread and the subtraction keeps its
// digits.  Two sets are combined after moving one onto the other's shift K':
//   S' = S + n (K - K'),  Q' = Q + (K - K') (2 S + n (K - K'))
// (plain multiply-adds: no division on the reduction's critical path).
// Two double2 slots of a partial-sum buffer hold one Moments.
struct __align__(16) Moments {
    double n, k, s, q;
};

__device__ __forceinline__ Moments mom_shift(const Moments &a, double k2)
{
    const double dk = a.k - k2;
    Moments r;
    r.n = a.n;
    r.k = k2;
    r.s = fma(a.n, dk, a.s);
    r.q = fma(dk, fma(a.n, dk, 2.0 * a.s), a.q);
    return r;
}

// mean and M2 of a set (n > 0)
__device__ __forceinline__ void mom_mean_m2(const Moments &a, double *mean, double *m2)
{
    const double md = a.s / a.n;
    *mean = a.k + md;
    const double q = fma(-a.s, md, a.q);
    *m2 = q > 0.0 ? q : (q == q ? 0.0 : q);   // keeps a NaN
}

// One thread's values, shifted by its first value, in the kernel's own precision T.
template <typename T>
struct MomAcc {
    int n = 0;
    T k = 0, s = 0, q = 0;
    __device__ __forceinline__ void add(T x)
    {
        if (n == 0)
            k = x;
        const T d = x - k;
        s += d;
        q = fma(d, d, q);
        ++n;
    }
};

// The same shifted sums in precision T, for the warp-level part of a block reduction
// (FP32 kernels keep it in FP32: on this part an FP64 instruction costs the issue
// slots of 64 FP32 ones).  n stays exact in FP32 up to 2^24 values a warp.
template <typename T>
struct MomT {
    T n, k, s, q;
};

template <typename T>
__device__ __forceinline__ MomT<T> momt_shift(const MomT<T> &a, T k2)
{
    const T dk = a.k - k2;
    return MomT<T>{a.n, k2, fma(a.n, dk, a.s), fma(dk, fma(a.n, dk, a.s + a.s), a.q)};
}

// Deterministic combination over the block, on the shift of thread 0 (which holds the
// block's first value whenever the block has any): each warp moves its lanes onto its
// lane 0's shift and sums them in T; warp 0 moves the warps onto warp 0's shift and
// sums them in FP64.  The result is valid in thread 0.  Every thread must call it.
template <typename T>
__device__ __forceinline__ Moments block_moments(const MomAcc<T> &acc)
{
    __shared__ Moments smem_mom[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    MomT<T> v{(T)acc.n, acc.k, acc.s, acc.q};
    v = momt_shift(v, __shfl_sync(0xffffffffu, v.k, 0));
    for (int o = 16; o > 0; o >>= 1) {
        v.n += __shfl_down_sync(0xffffffffu, v.n, o);
        v.s += __shfl_down_sync(0xffffffffu, v.s, o);
        v.q += __shfl_down_sync(0xffffffffu, v.q, o);
    }
    __syncthreads();
    if (lane == 0)
        smem_mom[w] = Moments{(double)v.n, (double)v.k, (double)v.s, (double)v.q};
    __syncthreads();
    Moments r{0.0, 0.0, 0.0, 0.0};
    if (w == 0) {
        const double kb = smem_mom[0].k;
        r = lane < nw ? mom_shift(smem_mom[lane], kb) : Moments{0.0, kb, 0.0, 0.0};
        for (int o = 16; o > 0; o >>= 1) {
            if (o >= nw)   // lanes >= nw hold zeros (uniform test)
                continue;
            r.n += __shfl_down_sync(0xffffffffu, r.n, o);
            r.s += __shfl_down_sync(0xffffffffu, r.s, o);
            r.q += __shfl_down_sync(0xffffffffu, r.q, o);
        }
    }
    return r;
}

// Sets that already share one shift k (the finalize): plain sums over the block in
// FP64; the result is valid in thread 0.  Every thread must call it.
__device__ __forceinline__ Moments block_sum_shared_shift(Moments v)
{
    __shared__ Moments smem_mss[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        v.n += __shfl_down_sync(0xffffffffu, v.n, o);
        v.s += __shfl_down_sync(0xffffffffu, v.s, o);
        v.q += __shfl_down_sync(0xffffffffu, v.q, o);
    }
    __syncthreads();
    if (lane == 0)
        smem_mss[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? smem_mss[lane] : Moments{0.0, v.k, 0.0, 0.0};
        for (int o = 16; o > 0; o >>= 1) {
            if (o >= nw)
                continue;
            v.n += __shfl_down_sync(0xffffffffu, v.n, o);
            v.s += __shfl_down_sync(0xffffffffu, v.s, o);
            v.q += __shfl_down_sync(0xffffffffu, v.q, o);
        }
    }
    return v;
}

// Deterministic sum of a double2 over the block; the result is valid in thread 0.
// Every thread of the block must call it.
__device__ __forceinline__ double2 block_sum2(double2 v)
{
    __shared__ double2 smem_sum2[32];
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0)
        smem_sum2[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < nw ? smem_sum2[lane] : make_double2(0.0, 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
    }
    return v;
}

}  // namespace mg5
