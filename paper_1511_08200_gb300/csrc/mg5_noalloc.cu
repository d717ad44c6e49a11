// mg5_noalloc.cu -- a residual-norm entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running under a memory pool or
// allocator it does not own, inside a region where allocation would
// synchronise the device or break an enclosing capture, or a host program
// that only hands out pointers to buffers it already owns.  For them, the
// reduction's per-block partial sums live in a fixed file-scope device array
// instead of context scratch.  The caller still passes every input and
// output.  The array is a host-side symbol: its device address is looked up
// once per device (cudaGetSymbolAddress) and the kernels are given that.
#include <cuda_runtime.h>

#include <mutex>

#include "mg5.h"
#include "mg5_kernels.cuh"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 4096;       // one Moments slot per block
constexpr int kNoAllocCellsPerThread = 2;     // N^3 <= 4096 * 256 * 2 = 2,097,152 (N <= 128)
constexpr int kNoAllocMaxDevices = 64;

// Shared by every call on a device and kept until the process exits (128 KiB); a call
// overwrites exactly the slots it reads, so nothing needs clearing.
static __device__ __align__(256) mg5::Moments g_noalloc_partials[kNoAllocMaxBlocks];

std::mutex g_noalloc_mu;
mg5::Moments *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// r = f + c - op(phi) on the periodic cube; per block the shifted sums of r
__global__ void k_residual_partials(const double *__restrict__ phi, const double *__restrict__ f,
                                    double c, int n, mg5::CoefT<double> cf, mg5::Moments *partials)
{
    using namespace mg5;
    const long long total = (long long)n * n * n;
    MomAcc<double> acc;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(t % n);
        const long long q = t / n;
        const int j = (int)(q % n), i = (int)(q / n);
        const Rows r = periodic_rows(n, i, j);
        const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
        St<double> s;
        gather(phi, phi, r, k, kp, km, s);
        acc.add(cell_residual(s, MG5_AT(f, t) + c, cf));
    }
    const Moments m = block_moments(acc);
    if (threadIdx.x == 0)
        MG5_AT(partials, blockIdx.x) = m;
}

// out[0] = mean r, out[1] = ||r - mean r||_2, out[2] = ||r||_2 from the blocks' shifted
// sums, moved onto block 0's shift and summed in a fixed order (no cancellation when
// |mean r| is far above its spread)
__global__ void k_norm_finalize(const mg5::Moments *__restrict__ partials, int nb, double *out)
{
    using namespace mg5;
    const double k0 = MG5_AT(partials, 0).k;
    Moments v{0.0, k0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const Moments u = mom_shift(MG5_AT(partials, b), k0);
        v.n += u.n;
        v.s += u.s;
        v.q += u.q;
    }
    v = block_sum_shared_shift(v);
    if (threadIdx.x == 0) {
        double m = 0.0, m2 = 0.0;
        if (v.n > 0.0)
            mom_mean_m2(v, &m, &m2);
        MG5_AT(out, 0) = m;
        MG5_AT(out, 1) = sqrt(m2);
        MG5_AT(out, 2) = sqrt(fma(v.n * m, m, m2));   // sum r^2 = M2 + n mean^2
    }
}

// Device address of this device's partial array, looked up once per device.
cudaError_t partials_address(mg5::Moments **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess)
            return e;
        g_noalloc_ptr[dev] = static_cast<mg5::Moments *>(p);
#ifdef MG5_BOUNDS
        mg5::bnd::note_range(p, sizeof(g_noalloc_partials));
#endif
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

long long mg5_residual_norm_noalloc_max_cells(void)
{
    return (long long)kNoAllocMaxBlocks * kNoAllocThreads * kNoAllocCellsPerThread;
}

int mg5_residual_norm_noalloc(const double *phi, const double *f, double c, int N, double h,
                              double alpha, double *out, void *stream)
{
    if (!phi || !f || !out || N < 1 || !(h > 0.0) || !(alpha >= 0.0))
        return MG5_E_ARG;
    const long long n3 = (long long)N * N * N;
    if (n3 > mg5_residual_norm_noalloc_max_cells())
        return MG5_E_TOO_LARGE;
    mg5::Moments *partials = nullptr;
    if (partials_address(&partials) != cudaSuccess) {
        cudaGetLastError();
        return MG5_E_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    long long nb = (n3 + kNoAllocThreads - 1) / kNoAllocThreads;
    if (nb > kNoAllocMaxBlocks)
        nb = kNoAllocMaxBlocks;
    k_residual_partials<<<(int)nb, kNoAllocThreads, 0, st>>>(phi, f, c, N,
                                                             mg5::make_coef<double>(h, alpha), partials);
    k_norm_finalize<<<1, 1024, 0, st>>>(partials, (int)nb, out);
    mg5::count_launch(2);
    return cudaGetLastError() == cudaSuccess ? MG5_OK : MG5_E_CUDA;
}

}  // extern "C"
