// mg5_fin.cuh -- the end of a residual or norm reduction, done by the last block of the
// producing kernel instead of a separate one-block launch.
//
// Every reduction kernel writes one partial per block (double2 sums, or Moments for the
// residual statistics).  With a Fin target, each block then counts itself done on a
// counter kept in the partial buffer's last slot; the block that counts last reads all
// partials (past L1: they were written by other SMs in this launch) and applies the
// finalize rule of its mode, then zeroes the counter for the next launch.  The partials
// are combined in block order, the same order as the one-block finalize kernel, so the
// result does not depend on which block finishes last.
#pragma once
#include "mg5_kernels.cuh"

namespace mg5 {

__device__ __forceinline__ unsigned *fin_counter(double2 *partials)
{
    return &MG5_AT(reinterpret_cast<unsigned *>(partials + kMaxPartials - 1), 0);
}

// Apply `mode` to nb partials (all threads of the block must call it).
__device__ __forceinline__ void finalize_body(const double2 *partials, int nb, double ncells,
                                              LevelScal *ls, int mode)
{
    ls = &MG5_AT(ls, 0);
    if (mode == FIN_RESID || mode == FIN_STATS) {
        // per-block shifted sums moved onto block 0's shift, summed in a fixed order
        auto ld = [&](int b) {
            const double2 u = __ldcg(&MG5_AT(partials, 2 * b)), w = __ldcg(&MG5_AT(partials, 2 * b + 1));
            return Moments{u.x, u.y, w.x, w.y};
        };
        const double k0 = ld(0).k;
        Moments v{0.0, k0, 0.0, 0.0};
        for (int b = threadIdx.x; b < nb; b += blockDim.x) {
            const Moments u = mom_shift(ld(b), k0);
            v.n += u.n;
            v.s += u.s;
            v.q += u.q;
        }
        v = block_sum_shared_shift(v);
        if (threadIdx.x != 0)
            return;
        double m = 0.0, m2 = 0.0;
        if (v.n > 0.0)
            mom_mean_m2(v, &m, &m2);
        ls->m = m;
        if (mode == FIN_RESID)
            ls->c -= m;
        ls->rnorm = sqrt(m2);
        ls->rel = ls->fnorm > 0.0 ? ls->rnorm / ls->fnorm : ls->rnorm;
        if (!isfinite(m) || !isfinite(m2))
            ls->rel = m + m2;  // propagates NaN / Inf to the host check
        return;
    }
    double2 acc = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double2 u = __ldcg(&MG5_AT(partials, b));
        acc.x += u.x;
        acc.y += u.y;
    }
    acc = block_sum2(acc);
    if (threadIdx.x != 0)
        return;
    if (mode == FIN_NORM) {
        ls->m = acc.x / ncells;
        ls->rnorm = sqrt(acc.y);
        ls->rel = ls->fnorm > 0.0 ? ls->rnorm / ls->fnorm : ls->rnorm;
        if (!isfinite(acc.x) || !isfinite(acc.y))
            ls->rel = acc.y + acc.x;
    } else if (mode == FIN_FNORM) {
        ls->fnorm = sqrt(acc.y);
    } else {
        ls->mean = acc.x / ncells;
    }
}

// Called by every thread of every block after thread 0 has written the block's partial.
// The partials are indexed by the linear block index (x fastest).
__device__ __forceinline__ void finalize_if_last(double2 *partials, const Fin &fin)
{
    __shared__ int s_last;
    const unsigned nblk = gridDim.x * gridDim.y * gridDim.z;
    if (threadIdx.x == 0) {
        __threadfence();   // the partial before the count
        s_last = atomicAdd(fin_counter(partials), 1u) == nblk - 1;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    finalize_body(partials, (int)nblk, fin.ncells, fin.ls, fin.mode);
    if (threadIdx.x == 0)
        *fin_counter(partials) = 0u;
}

}  // namespace mg5
