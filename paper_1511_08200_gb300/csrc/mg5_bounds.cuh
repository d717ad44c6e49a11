// mg5_bounds.cuh -- the range-checked build (-DMG5_BOUNDS, libmg5_bounds.so).
//
// Every global-memory element a kernel reads or writes through MG5_AT(p, i) is checked
// against the device allocations the library knows: its own (each cudaMalloc of the
// library's host code registers its range) and the caller's buffers (the containing
// allocation of each pointer handed to the library, noted through mg5_bounds_note).
// Shared-memory elements reached through a generic pointer are checked against the CTA's
// shared-memory size, and the 16-byte asynchronous copies check both ends.  A violation
// does not trap: the access goes to a scratch word instead (a copy is skipped), and the
// first violation of a translation unit is kept in a device error word (the line of the
// access and its kind: 1 global, 2 shared, 3 copy source, 4 copy destination) that
// mg5_bounds_check() reads and clears.  Local-memory addresses pass unchecked.
//
// In the ordinary build MG5_AT(p, i) is p[i] and nothing below exists.
#pragma once
#include <cuda_runtime.h>

#ifdef MG5_BOUNDS

namespace mg5 {
namespace bnd {

constexpr int kRanges = 1024;   // allocations tracked at once

struct Table {
    int n;
    int pad;
    unsigned long long lo[kRanges];
    unsigned long long hi[kRanges];   // one past the last byte
};

// host side (mg5_bounds.cu): the per-translation-unit hooks and the range registry
struct TuHooks {
    const char *name;
    cudaError_t (*upload)(const void *src, size_t bytes, size_t offset);   // into the table
    unsigned long long (*take_error)();
};
void register_tu(const TuHooks &h);
cudaError_t note_range(const void *p, size_t bytes);
void forget_range(const void *p);
cudaError_t malloc_checked(void **p, size_t bytes);
cudaError_t free_checked(void *p);

namespace {

__device__ Table g_table;
__device__ unsigned long long g_error;   // (line << 8) | kind of the first violation
__device__ double4 g_scratch[2];         // where a rejected access goes

__device__ __noinline__ void violation(int line, int kind)
{
    atomicCAS(&g_error, 0ull, ((unsigned long long)line << 8) | (unsigned long long)kind);
}

__device__ __forceinline__ bool global_ok(unsigned long long a, unsigned long long bytes)
{
    const int n = g_table.n;
    for (int r = 0; r < n; ++r)
        if (a >= g_table.lo[r] && a + bytes <= g_table.hi[r])
            return true;
    return false;
}

__device__ __forceinline__ bool shared_ok(const void *q, unsigned bytes)
{
    unsigned total;
    asm volatile("mov.u32 %0, %%total_smem_size;" : "=r"(total));
    const unsigned off = (unsigned)__cvta_generic_to_shared(q);
    // 1 KiB of the window below the CTA's own shared memory is reserved on sm_90 and later
    return off + bytes <= total + 1024u;
}

template <typename T>
__device__ __forceinline__ T *at(T *p, long long i, int line)
{
    T *q = p + i;
    if (__isShared(q)) {
        if (shared_ok(q, sizeof(T)))
            return q;
        violation(line, 2);
    } else if (__isLocal(q)) {
        return q;
    } else {
        if (global_ok((unsigned long long)q, sizeof(T)))
            return q;
        violation(line, 1);
    }
    return reinterpret_cast<T *>(g_scratch);
}

// the two ends of a 16-byte global -> shared copy: false when the copy must be skipped
__device__ __forceinline__ bool copy_ok(unsigned smem, const void *g, int line)
{
    unsigned total;
    asm volatile("mov.u32 %0, %%total_smem_size;" : "=r"(total));
    if (smem + 16u > total + 1024u) {
        violation(line, 4);
        return false;
    }
    if (!global_ok((unsigned long long)g, 16)) {
        violation(line, 3);
        return false;
    }
    return true;
}

cudaError_t tu_upload(const void *src, size_t bytes, size_t offset)
{
    return cudaMemcpyToSymbol(g_table, src, bytes, offset);
}

unsigned long long tu_take_error()
{
    unsigned long long e = 0, z = 0;
    if (cudaMemcpyFromSymbol(&e, g_error, sizeof(e)) != cudaSuccess)
        return 0;
    if (e)
        cudaMemcpyToSymbol(g_error, &z, sizeof(z));
    return e;
}

struct TuRegistrar {
    TuRegistrar() { register_tu(TuHooks{__BASE_FILE__, tu_upload, tu_take_error}); }
};
TuRegistrar g_tu_registrar;

}  // namespace
}  // namespace bnd
}  // namespace mg5

#define MG5_AT(p, i) (*::mg5::bnd::at((p), (long long)(i), __LINE__))

// the library's own device allocations register their ranges
#ifndef MG5_BOUNDS_IMPL
#define cudaMalloc(p, b) ::mg5::bnd::malloc_checked((void **)(p), (size_t)(b))
#define cudaFree(p) ::mg5::bnd::free_checked((void *)(p))
#endif

#else

#define MG5_AT(p, i) ((p)[i])

#endif
