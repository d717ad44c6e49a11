// mg5_async.cuh -- small helpers of the plane-marching kernels: 16-byte asynchronous
// global -> shared copies (cp.async, completion tracked per thread by commit groups) and
// the periodic wrap of an index that is at most one period out of range.
#pragma once
#include <cuda_runtime.h>

#include "mg5_bounds.cuh"

namespace mg5 {
namespace acopy {

__device__ __forceinline__ void copy16(unsigned smem_addr, const void *gmem)
{
#ifdef MG5_BOUNDS
    if (!::mg5::bnd::copy_ok(smem_addr, gmem, __LINE__))
        return;
#endif
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace acopy

__device__ __forceinline__ int wrap_once(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

}  // namespace mg5
