// k_mask.cu -- kernels of the position-dependent truncation (Sec. 3.3).
//
// For screening that does not follow the refinement structure, Sec. 3.3 sketches a
// criterion per cell: iterate a fine cell of level l+1 only while the fifth force on
// its parent (the level-l cell that was refined) is still large.  A refinement then
// relaxes a subset of its cells, given as a byte mask over the patch interior; the
// other cells keep the values interpolated from the parent and act as fixed
// neighbours.  These kernels build that mask from the parent level's forces, carry
// it down the patch's multigrid hierarchy, and form the masked source norm.
#include "mg5_kernels.cuh"

namespace mg5 {

// mc(I, J, K) = AND of the 8 children (2I + a, 2J + b, 2K + c) of the fine mask.  A coarse
// cell is relaxed only when all its children are: a cell with some children held fixed would
// solve a coarse equation for a change of all 8 children while only some of them take it, and
// that inconsistency made the V-cycle diverge (a linear model of the masked cycle grew by 1.6
// per cycle with the OR rule and contracted by 0.08 - 0.14 with this one).  Cells at the edge
// of the masked region are left to the fine-grid sweeps.
__global__ void k_mask_restrict(const unsigned char *__restrict__ mf, int p0, int p1, int p2,
                                unsigned char *__restrict__ mc)
{
    const int q0 = p0 >> 1, q1 = p1 >> 1, q2 = p2 >> 1;
    const long long total = (long long)q0 * q1 * q2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total)
        return;
    const int K = (int)(t % q2);
    const long long q = t / q2;
    const int J = (int)(q % q1), I = (int)(q / q1);
    unsigned char all = 1;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        const int i = 2 * I + (ch >> 2), j = 2 * J + ((ch >> 1) & 1), k = 2 * K + (ch & 1);
        all &= MG5_AT(mf, ((long long)i * p1 + j) * p2 + k) ? 1 : 0;
    }
    MG5_AT(mc, t) = all;
}

cudaError_t launch_mask_restrict(const unsigned char *mf, const int p[3], unsigned char *mc,
                                 cudaStream_t st)
{
    const long long work = (long long)(p[0] / 2) * (p[1] / 2) * (p[2] / 2);
    k_mask_restrict<<<blocks_for(work), kBlock, 0, st>>>(mf, p[0], p[1], p[2], mc);
    count_launch(1);
    return cudaGetLastError();
}

// f = s delta + add on every cell; partial sums (number of masked cells, (s delta)^2 over them)
__global__ void k_scale_masked(const double *__restrict__ delta, double s, double *__restrict__ f,
                               long long n, const unsigned char *__restrict__ mask,
                               double2 *__restrict__ partials, double add)
{
    double2 acc = make_double2(0.0, 0.0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const double v = s * MG5_AT(delta, t);
        MG5_AT(f, t) = v + add;
        if (MG5_AT(mask, t)) {
            acc.x += 1.0;
            acc.y += v * v;
        }
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = acc;
}

cudaError_t launch_scale_masked(const double *delta, double s, double *f, long long n,
                                const unsigned char *mask, double2 *partials, int *nblocks,
                                cudaStream_t st, double add)
{
    int g = blocks_for(n);
    if (g > kReduceBlocks)
        g = kReduceBlocks;
    k_scale_masked<<<g, kBlock, 0, st>>>(delta, s, f, n, mask, partials, add);
    *nblocks = g;
    count_launch(1);
    return cudaGetLastError();
}

// One thread per fine interior cell of the (2 pn) patch: its parent is cell
// (o + I/2, o + J/2, o + K/2) of the parent grid of dims pd (wrapped when periodic);
// F5 = grad(phi)/2 (Sec. 3.2), F_GR = grad(Psi_GR), both SoA (3 blocks of the parent's
// cells).  mask = |F5| > theta |F_GR| (no division: a parent with F_GR = 0 is iterated where
// F5 != 0); products and sums rounded one by one (no fused multiply-add), so the decision is
// the plain IEEE one.  `count` accumulates the masked cells.
__global__ void k_parent_force_mask(const double *__restrict__ gphi, const double *__restrict__ ggr,
                                    int pd0, int pd1, int pd2, int periodic, int o0, int o1, int o2,
                                    int P0, int P1, int P2, double theta,
                                    unsigned char *__restrict__ mask, unsigned long long *count)
{
    const long long total = (long long)P0 * P1 * P2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool on = false;
    if (t < total) {
        const int K = (int)(t % P2);
        const long long q = t / P2;
        const int J = (int)(q % P1), I = (int)(q / P1);
        int ci = o0 + (I >> 1), cj = o1 + (J >> 1), ck = o2 + (K >> 1);
        if (periodic) {
            ci -= ci >= pd0 ? pd0 : 0;
            cj -= cj >= pd1 ? pd1 : 0;
            ck -= ck >= pd2 ? pd2 : 0;
        }
        const long long n3 = (long long)pd0 * pd1 * pd2;
        const long long pc = ((long long)ci * pd1 + cj) * pd2 + ck;
        double f5 = 0.0, fg = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x = 0.5 * MG5_AT(gphi, a * n3 + pc), y = MG5_AT(ggr, a * n3 + pc);
            f5 = __dadd_rn(f5, __dmul_rn(x, x));
            fg = __dadd_rn(fg, __dmul_rn(y, y));
        }
        on = sqrt(f5) > __dmul_rn(theta, sqrt(fg));
        MG5_AT(mask, t) = on ? 1 : 0;
    }
    if (count) {
        const unsigned ballot = __ballot_sync(0xffffffffu, on);
        if ((threadIdx.x & 31) == 0 && ballot)
            atomicAdd(&MG5_AT(count, 0), (unsigned long long)__popc(ballot));
    }
}

cudaError_t launch_parent_force_mask(const double *grad_phi, const double *grad_gr, const int pd[3],
                                     int periodic, const int o[3], const int pn[3], double theta,
                                     unsigned char *mask, unsigned long long *count,
                                     cudaStream_t st)
{
    const long long work = 8ll * pn[0] * pn[1] * pn[2];
    k_parent_force_mask<<<blocks_for(work), kBlock, 0, st>>>(
        grad_phi, grad_gr, pd[0], pd[1], pd[2], periodic ? 1 : 0, o[0], o[1], o[2], 2 * pn[0],
        2 * pn[1], 2 * pn[2], theta, mask, count);
    count_launch(1);
    return cudaGetLastError();
}

}  // namespace mg5
