// mg5_bounds.cu -- host side of the range-checked build (mg5_bounds.cuh): the registry of
// device allocations the kernels may touch, mirrored into every translation unit's device
// table, and the C entry points that note caller buffers and report violations.  In the
// ordinary build the entry points exist and do nothing.
#define MG5_BOUNDS_IMPL
#include "mg5_bounds.cuh"

#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "mg5.h"

#ifdef MG5_BOUNDS

namespace mg5 {
namespace bnd {
namespace {

std::mutex &mu()
{
    static std::mutex m;
    return m;
}
std::vector<TuHooks> &tus()
{
    static std::vector<TuHooks> v;
    return v;
}
Table &table()
{
    static Table t{};
    return t;
}
// which entries are caller buffers (evicted first when the table is full)
std::vector<char> &is_caller()
{
    static std::vector<char> v(kRanges, 0);
    return v;
}

// entry r, then the count: a kernel reading the table meanwhile sees either state
cudaError_t upload_entry(int r)
{
    const Table &t = table();
    for (const TuHooks &h : tus()) {
        cudaError_t e = h.upload(&t.lo[r], sizeof(t.lo[r]), offsetof(Table, lo) + r * sizeof(t.lo[0]));
        if (e == cudaSuccess)
            e = h.upload(&t.hi[r], sizeof(t.hi[r]), offsetof(Table, hi) + r * sizeof(t.hi[0]));
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t upload_count()
{
    const Table &t = table();
    for (const TuHooks &h : tus()) {
        cudaError_t e = h.upload(&t.n, sizeof(t.n), offsetof(Table, n));
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t add_locked(unsigned long long lo, unsigned long long hi, bool caller)
{
    Table &t = table();
    for (int r = 0; r < t.n; ++r)
        if (lo >= t.lo[r] && hi <= t.hi[r])
            return cudaSuccess;
    int r = t.n;
    if (r == kRanges) {   // full: reuse the slot of a caller buffer
        r = -1;
        for (int q = 0; q < t.n; ++q)
            if (is_caller()[q]) {
                r = q;
                break;
            }
        if (r < 0) {
            std::fprintf(stderr, "mg5 bounds: more than %d device allocations\n", kRanges);
            return cudaErrorMemoryAllocation;
        }
    }
    t.lo[r] = lo;
    t.hi[r] = hi;
    is_caller()[r] = caller ? 1 : 0;
    cudaError_t e = upload_entry(r);
    if (e == cudaSuccess && r == t.n) {
        ++t.n;
        e = upload_count();
    }
    return e;
}

}  // namespace

void register_tu(const TuHooks &h)
{
    std::lock_guard<std::mutex> g(mu());
    tus().push_back(h);
}

cudaError_t note_range(const void *p, size_t bytes)
{
    std::lock_guard<std::mutex> g(mu());
    const unsigned long long lo = (unsigned long long)p;
    return add_locked(lo, lo + bytes, false);
}

void forget_range(const void *p)
{
    std::lock_guard<std::mutex> g(mu());
    Table &t = table();
    const unsigned long long a = (unsigned long long)p;
    for (int r = 0; r < t.n; ++r)
        if (t.lo[r] == a) {
            const int last = t.n - 1;
            if (r != last) {   // the last entry moves into r, then the count drops
                t.lo[r] = t.lo[last];
                t.hi[r] = t.hi[last];
                is_caller()[r] = is_caller()[last];
                upload_entry(r);
            }
            t.n = last;
            upload_count();
            return;
        }
}

cudaError_t malloc_checked(void **p, size_t bytes)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess)
        e = note_range(*p, bytes);
    return e;
}

cudaError_t free_checked(void *p)
{
    // cudaFree waits for the device first, so no kernel still uses the range it drops
    cudaError_t e = cudaFree(p);
    if (p)
        forget_range(p);
    return e;
}

}  // namespace bnd
}  // namespace mg5

extern "C" {

int mg5_bounds_build(void) { return 1; }

int mg5_bounds_note(const void *p)
{
    if (!p)
        return MG5_OK;
    using GetRange = int (*)(unsigned long long *, size_t *, unsigned long long);
    static GetRange get_range = nullptr;
    if (!get_range) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return MG5_E_CUDA;
        get_range = reinterpret_cast<GetRange>(fn);
    }
    unsigned long long base = 0;
    size_t size = 0;
    if (get_range(&base, &size, (unsigned long long)p) != 0)
        return MG5_E_ARG;   // not device memory
    std::lock_guard<std::mutex> g(mg5::bnd::mu());
    return mg5::bnd::add_locked(base, base + size, true) == cudaSuccess ? MG5_OK : MG5_E_CUDA;
}

int mg5_bounds_check(char *msg, int cap)
{
    std::lock_guard<std::mutex> g(mg5::bnd::mu());
    int found = 0;
    for (const mg5::bnd::TuHooks &h : mg5::bnd::tus()) {
        const unsigned long long e = h.take_error();
        if (e && !found) {
            found = 1;
            if (msg && cap > 0) {
                static const char *kinds[] = {"?", "global element", "shared element",
                                              "copy source", "copy destination"};
                const int kind = (int)(e & 0xff);
                std::snprintf(msg, (size_t)cap, "%s: line %llu: %s out of range", h.name,
                              e >> 8, kinds[kind >= 1 && kind <= 4 ? kind : 0]);
            }
        }
    }
    return found;
}

}  // extern "C"

#else

extern "C" {
int mg5_bounds_build(void) { return 0; }
int mg5_bounds_note(const void *) { return MG5_OK; }
int mg5_bounds_check(char *msg, int cap)
{
    if (msg && cap > 0)
        msg[0] = 0;
    return 0;
}
}

#endif
