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
constexpr int kNoAllocMaxBlocks = 8192;   // one block per 256 cells: N^3 <= 2,097,152 (N <= 128)
constexpr int kNoAllocMaxDevices = 64;

// Shared by every call on a device and kept until the process exits; a call
// overwrites exactly the slots it reads, so nothing needs clearing.
static __device__ __align__(256) double2 g_noalloc_partials[kNoAllocMaxBlocks];

std::mutex g_noalloc_mu;
double2 *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// r = f + c - op(phi) on the periodic cube; block partial sums (sum r, sum r^2)
__global__ void k_residual_partials(const double *__restrict__ phi, const double *__restrict__ f,
                                    double c, int n, mg5::CoefT<double> cf, double2 *partials)
{
    using namespace mg5;
    const long long total = (long long)n * n * n;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double2 acc = make_double2(0.0, 0.0);
    if (t < total) {
        const int k = (int)(t % n);
        const long long q = t / n;
        const int j = (int)(q % n), i = (int)(q / n);
        const Rows r = periodic_rows(n, i, j);
        const int kp = (k == n - 1) ? 0 : k + 1, km = (k == 0) ? n - 1 : k - 1;
        St<double> s;
        gather(phi, phi, r, k, kp, km, s);
        const double res = f[t] + c - cell_op(s, cf);
        acc.x = res;
        acc.y = res * res;
    }
    acc = block_sum2(acc);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = acc;
}

// out[0] = mean r, out[1] = ||r - mean r||_2, out[2] = ||r||_2 (fixed summation order)
__global__ void k_norm_finalize(const double2 *__restrict__ partials, int nb, double ncells,
                                double *out)
{
    double2 acc = make_double2(0.0, 0.0);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        acc.x += partials[b].x;
        acc.y += partials[b].y;
    }
    acc = mg5::block_sum2(acc);
    if (threadIdx.x == 0) {
        const double m = acc.x / ncells;
        const double q2 = acc.y - ncells * m * m;
        out[0] = m;
        out[1] = sqrt(q2 > 0.0 ? q2 : 0.0);
        out[2] = sqrt(acc.y);
    }
}

// Device address of this device's partial-sum array, looked up once per device.
cudaError_t partials_address(double2 **out)
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
        g_noalloc_ptr[dev] = static_cast<double2 *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" {

long long mg5_residual_norm_noalloc_max_cells(void)
{
    return (long long)kNoAllocMaxBlocks * kNoAllocThreads;
}

int mg5_residual_norm_noalloc(const double *phi, const double *f, double c, int N, double h,
                              double alpha, double *out, void *stream)
{
    if (!phi || !f || !out || N < 1 || !(h > 0.0) || !(alpha >= 0.0))
        return MG5_E_ARG;
    const long long n3 = (long long)N * N * N;
    if (n3 > mg5_residual_norm_noalloc_max_cells())
        return MG5_E_TOO_LARGE;
    double2 *partials = nullptr;
    if (partials_address(&partials) != cudaSuccess) {
        cudaGetLastError();
        return MG5_E_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)((n3 + kNoAllocThreads - 1) / kNoAllocThreads);
    k_residual_partials<<<nb, kNoAllocThreads, 0, st>>>(phi, f, c, N, mg5::make_coef<double>(h, alpha),
                                                        partials);
    k_norm_finalize<<<1, 1024, 0, st>>>(partials, nb, (double)n3, out);
    mg5::count_launch(2);
    return cudaGetLastError() == cudaSuccess ? MG5_OK : MG5_E_CUDA;
}

}  // extern "C"
