// k_bottom.cu -- the bottom of a V-cycle in one CTA: the visit of the grid a just above the
// coarsest grid b (side na <= 8, nb = na / 2) together with the solve of b, with the same
// steps, in the same order and with the same cell arithmetic as the level-by-level
// launches (Sec. 3.1: FAS coarse right-hand side, nu1 snapshot red-black sweeps, residual
// with its mean subtracted from the compatibility constant, 8-child restriction, the
// coarsest-grid iteration, trilinear prolongation of the correction, nu2 sweeps).  On these
// grids every launch costs more than its cells, so the thirteen-odd launches of a visit
// become one; the grids live in shared memory, one thread per cell of a.
//
// The mixed mode's FP32 inner solve uses it (the 128^3 mixed solve went 7.6 -> 6.6 ms, the
// launches of a step fell by a sixth).  The FP64 solves keep the launches: FP64 runs at 2
// lanes per clock on an SM, and the visit on one SM was slower than the launches spread over
// several (the 32^3 FP64 solve went 1.49 -> 1.65 ms with it).
//
// On entry v_a = R v (the restricted iterate of the grid above) and f_a = R r; on exit v_a
// holds the corrected iterate and the level scalars of a its constant c and residual mean m,
// which the launch that prolongs a's correction upward reads.  Periodic grids; with a base
// (the mixed mode's correction form) B_a and B_b are the restricted bases.
#include "mg5_fin.cuh"

namespace mg5 {

namespace {

constexpr int kBottomMax = 8;                               // largest side of grid a
constexpr int kBottomThreads = kBottomMax * kBottomMax * kBottomMax;

// smem: a: v, w (sweep partner), f, r (residual scratch), B; b: v, w, f, v0, B
template <typename T>
struct BottomSmem {
    T av[kBottomThreads], aw[kBottomThreads], af[kBottomThreads], ar[kBottomThreads],
        aB[kBottomThreads];
    T bv[kBottomThreads / 8], bw[kBottomThreads / 8], bf[kBottomThreads / 8],
        b0[kBottomThreads / 8], bB[kBottomThreads / 8];
};

// one snapshot red-black sweep over the cells this thread owns (one cell, or none), v <-> w
template <typename T, bool BASE>
__device__ __forceinline__ void bsweep(T *v, T *w, const T *f, const T *B, bool mine, int p,
                                       const Nbr &nb, int colour_me, T c, const CoefT<T> &cf,
                                       unsigned long long &clamps)
{
    for (int colour = 0; colour < 2; ++colour) {
        const T *src = colour == 0 ? v : w;
        T *dst = colour == 0 ? w : v;
        if (mine) {
            if (colour_me != colour) {
                MG5_AT(dst, p) = MG5_AT(src, p);
            } else {
                St<T> s, sb;
                gather_nbr(src, nb, s);
                if constexpr (BASE)
                    gather_nbr(B, nb, sb);
                bool cl = false;
                MG5_AT(dst, p) = upd<T, BASE>(s, sb, MG5_AT(f, p) + c, cf, cl);
                clamps += cl ? 1ull : 0ull;
            }
        }
        __syncthreads();
    }
}

// the coarsest grid (at most 64 cells) is iterated by the first two warps alone: a barrier
// over those 64 threads and their sum of a double2 (fixed order: warp 0, then warp 1)
__device__ __forceinline__ void bar64() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

__device__ __forceinline__ double2 sum64(double2 v, double2 *sm)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if ((threadIdx.x & 31) == 0)
        sm[threadIdx.x >> 5] = v;
    bar64();
    const double2 r = make_double2(sm[0].x + sm[1].x, sm[0].y + sm[1].y);
    bar64();
    return r;
}

template <typename T, bool BASE>
__device__ __forceinline__ void bsweep64(T *v, T *w, const T *f, const T *B, bool mine, int p,
                                         const Nbr &nb, int colour_me, T c, const CoefT<T> &cf,
                                         unsigned long long &clamps)
{
    for (int colour = 0; colour < 2; ++colour) {
        const T *src = colour == 0 ? v : w;
        T *dst = colour == 0 ? w : v;
        if (mine) {
            if (colour_me != colour) {
                MG5_AT(dst, p) = MG5_AT(src, p);
            } else {
                St<T> s, sb;
                gather_nbr(src, nb, s);
                if constexpr (BASE)
                    gather_nbr(B, nb, sb);
                bool cl = false;
                MG5_AT(dst, p) = upd<T, BASE>(s, sb, MG5_AT(f, p) + c, cf, cl);
                clamps += cl ? 1ull : 0ull;
            }
        }
        bar64();
    }
}

template <typename T, bool BASE>
__global__ void __launch_bounds__(kBottomThreads)
    k_bottom(T *__restrict__ va_g, const T *__restrict__ fa_g, const T *__restrict__ Ba_g,
             const T *__restrict__ Bb_g, int na, CoefT<T> cfa, CoefT<T> cfb,
             const LevelScal *__restrict__ ls_up, LevelScal *__restrict__ lsa,
             LevelScal *__restrict__ lsb, int nu1, int nu2, int nu_coarse, double rtol,
             unsigned long long *clamp, int *sweeps_out)
{
    __shared__ BottomSmem<T> S;
    __shared__ double bc_s[2];
    __shared__ double2 s64[2];
    const int nb = na >> 1;
    const int na3 = na * na * na, nb3 = nb * nb * nb;
    const int p = threadIdx.x;
    const bool mine = p < na3, mine_b = p < nb3;
    unsigned long long clamps = 0;

    // grid a: load, stencil offsets, colour
    Nbr nbr{};
    int colour_me = 0;
    if (mine) {
        S.av[p] = MG5_AT(va_g, p);
        S.af[p] = MG5_AT(fa_g, p);
        if constexpr (BASE)
            S.aB[p] = MG5_AT(Ba_g, p);
        const int k = p % na, j = (p / na) % na, i = p / (na * na);
        const int kp = (k == na - 1) ? 0 : k + 1, km = (k == 0) ? na - 1 : k - 1;
        nbr = nbr_of(periodic_rows(na, i, j), k, kp, km);
        colour_me = (i + j + k) & 1;
    }
    Nbr nbr_b{};
    int colour_b = 0;
    if (mine_b) {
        if constexpr (BASE)
            S.bB[p] = MG5_AT(Bb_g, p);
        const int k = p % nb, j = (p / nb) % nb, i = p / (nb * nb);
        const int kp = (k == nb - 1) ? 0 : k + 1, km = (k == 0) ? nb - 1 : k - 1;
        nbr_b = nbr_of(periodic_rows(nb, i, j), k, kp, km);
        colour_b = (i + j + k) & 1;
    }
    __syncthreads();

    // FAS right-hand side of a: f_a = op(v_a) + R r - m of the grid above; c_a = 0
    const double m_up = MG5_AT(ls_up, 0).m;
    if (mine) {
        St<T> s, sb;
        gather_nbr((const T *)S.av, nbr, s);
        if constexpr (BASE) {
            gather_nbr((const T *)S.aB, nbr, sb);
            S.af[p] = opr<T, BASE>(s, sb, cfa) + S.af[p] - (T)m_up;
        } else {
            S.af[p] = -cell_residual(s, (T)m_up - S.af[p], cfa);
        }
    }
    __syncthreads();
    double ca = 0.0;
    for (int it = 0; it < nu1; ++it)
        bsweep<T, BASE>(S.av, S.aw, S.af, S.aB, mine, p, nbr, colour_me, (T)ca, cfa, clamps);

    // residual of a, its mean (c_a -= m_a), and the 8-child restriction onto b
    double2 acc = make_double2(0.0, 0.0);
    if (mine) {
        St<T> s, sb;
        gather_nbr((const T *)S.av, nbr, s);
        if constexpr (BASE)
            gather_nbr((const T *)S.aB, nbr, sb);
        const T r = resid_of<T, BASE>(s, sb, S.af[p] + (T)ca, cfa);
        S.ar[p] = r;
        acc.x = (double)r;
    }
    acc = block_sum2(acc);
    if (p == 0)
        bc_s[0] = acc.x;
    __syncthreads();
    const double m_a = bc_s[0] / (double)na3;
    ca -= m_a;
    if (mine_b) {
        const int K = p % nb, J = (p / nb) % nb, I = p / (nb * nb);
        T sv = 0, sr = 0;
        for (int ch = 0; ch < 8; ++ch) {
            const int i = 2 * I + (ch >> 2), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch & 1);
            const int q = (i * na + j) * na + k;
            sv += S.av[q];
            sr += S.ar[q];
        }
        const T mv = sv * (T)0.125;
        S.bv[p] = mv;
        S.b0[p] = mv;
        S.bf[p] = sr * (T)0.125;
    }
    __syncthreads();

    // FAS right-hand side of b, then the coarsest-grid iteration (as k_coarsest)
    if (mine_b) {
        St<T> s, sb;
        gather_nbr((const T *)S.bv, nbr_b, s);
        if constexpr (BASE) {
            gather_nbr((const T *)S.bB, nbr_b, sb);
            S.bw[p] = opr<T, BASE>(s, sb, cfb) + S.bf[p] - (T)m_a;
        } else {
            S.bw[p] = -cell_residual(s, (T)m_a - S.bf[p], cfb);
        }
    }
    __syncthreads();
    if (mine_b)
        S.bf[p] = S.bw[p];
    __syncthreads();
    const double inv_nb3 = 1.0 / (double)nb3;
    double r0 = -1.0, cb = 0.0;
    int it = 0;
    if (p < 64) {
        for (; it < nu_coarse; ++it) {
            double2 a2 = make_double2(0.0, 0.0);
            if (mine_b) {
                St<T> s, sb;
                gather_nbr((const T *)S.bv, nbr_b, s);
                if constexpr (BASE)
                    gather_nbr((const T *)S.bB, nbr_b, sb);
                const double res = (double)resid_of<T, BASE>(s, sb, S.bf[p], cfb);
                a2.x = res;
                a2.y = res * res;
            }
            a2 = sum64(a2, s64);
            const double m = a2.x * inv_nb3;
            const double q2 = a2.y - (double)nb3 * m * m;
            const double rn = sqrt(q2 > 0.0 ? q2 : 0.0);
            cb = -m;
            if (r0 < 0.0)
                r0 = rn;
            if (rn <= rtol * r0)
                break;
            bsweep64<T, BASE>(S.bv, S.bw, S.bf, S.bB, mine_b, p, nbr_b, colour_b, (T)cb, cfb,
                              clamps);
        }
        if (p == 0)
            bc_s[1] = cb;
    }
    __syncthreads();
    cb = bc_s[1];

    // prolongation of b's correction onto a (cell-centred trilinear, periodic), c_a += c_b
    if (mine) {
        const int k = p % na, j = (p / na) % na, i = p / (na * na);
        const int I = i >> 1, J = j >> 1, K = k >> 1;
        const int I2 = (i & 1) ? (I + 1 == nb ? 0 : I + 1) : (I == 0 ? nb - 1 : I - 1);
        const int J2 = (j & 1) ? (J + 1 == nb ? 0 : J + 1) : (J == 0 ? nb - 1 : J - 1);
        const int K2 = (k & 1) ? (K + 1 == nb ? 0 : K + 1) : (K == 0 ? nb - 1 : K - 1);
        auto e = [&](int a, int b, int c) {
            const int q = (a * nb + b) * nb + c;
            return S.bv[q] - S.b0[q];
        };
        // weights (3/4, 1/4) per axis as 3x + y, one 1/64 at the end (as k_prolong_add)
        const T z00 = fma((T)3, e(I, J, K), e(I, J, K2)), z01 = fma((T)3, e(I, J2, K), e(I, J2, K2));
        const T z10 = fma((T)3, e(I2, J, K), e(I2, J, K2)), z11 = fma((T)3, e(I2, J2, K), e(I2, J2, K2));
        const T y0 = fma((T)3, z00, z01), y1 = fma((T)3, z10, z11);
        const T o = fma((T)3, y0, y1);
        S.av[p] = fma(o, (T)(1.0 / 64.0), S.av[p]);
    }
    ca += cb;
    __syncthreads();
    for (int s = 0; s < nu2; ++s)
        bsweep<T, BASE>(S.av, S.aw, S.af, S.aB, mine, p, nbr, colour_me, (T)ca, cfa, clamps);

    if (mine)
        MG5_AT(va_g, p) = S.av[p];
    if (clamps)
        atomicAdd(&MG5_AT(clamp, 0), clamps);
    if (p == 0) {
        LevelScal &A = MG5_AT(lsa, 0);
        A.m = m_a;
        A.c = ca;
        MG5_AT(lsb, 0).c = cb;
        if (sweeps_out)
            atomicAdd(&MG5_AT(sweeps_out, 0), it);
    }
}

}  // namespace

bool bottom_ok(int na) { return na >= 2 && na <= kBottomMax && na % 2 == 0; }

template <typename T>
cudaError_t launch_bottom(T *va, const T *fa, const T *Ba, const T *Bb, int na, CoefT<T> cfa,
                          CoefT<T> cfb, const LevelScal *ls_up, LevelScal *lsa, LevelScal *lsb,
                          int nu1, int nu2, int nu_coarse, double rtol, unsigned long long *clamp,
                          int *sweeps, cudaStream_t st)
{
    if (!bottom_ok(na) || (Ba == nullptr) != (Bb == nullptr))
        return cudaErrorInvalidValue;
    if (Ba)
        k_bottom<T, true><<<1, kBottomThreads, 0, st>>>(va, fa, Ba, Bb, na, cfa, cfb, ls_up, lsa,
                                                        lsb, nu1, nu2, nu_coarse, rtol, clamp,
                                                        sweeps);
    else
        k_bottom<T, false><<<1, kBottomThreads, 0, st>>>(va, fa, Ba, Bb, na, cfa, cfb, ls_up, lsa,
                                                         lsb, nu1, nu2, nu_coarse, rtol, clamp,
                                                         sweeps);
    count_launch(1);
    return cudaGetLastError();
}

template cudaError_t launch_bottom<float>(float *, const float *, const float *, const float *, int,
                                          CoefT<float>, CoefT<float>, const LevelScal *,
                                          LevelScal *, LevelScal *, int, int, int, double,
                                          unsigned long long *, int *, cudaStream_t);

}  // namespace mg5
