// kdss_internal.cuh -- shared internals of the CUDA solver (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "kdss.h"

namespace kdss {

// ---------------------------------------------------------------------------
// Errors: C++ exceptions inside the library, converted to kdss_status at the
// ABI boundary (api.cu).  Nothing throws across extern "C".
// ---------------------------------------------------------------------------
struct Error {
    kdss_status code;
    std::string msg;
};

[[noreturn]] void fail(kdss_status code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what, const char *file, int line);

#define KDSS_CUDA(call) ::kdss::check_cuda((call), #call, __FILE__, __LINE__)
// Arrays a caller passes as device memory must be device (or managed) memory
// of the device the work runs on (`dev`; -1: the current device) from their
// first to their last byte: the kernels would fault on a host pointer and
// write another device's memory through a peer pointer.  Throws INVALID_ARG,
// naming `what`, before any launch.
void check_device_array(const void *p, size_t bytes, const char *what, int dev = -1);
// Every kernel launch is followed by KDSS_LAUNCH_CHECK(), which also counts it.
void count_launch();
long long launches();               // kernels launched so far (process-wide)
long long thread_launches();        // kernels launched so far by the calling thread
void add_launches(long long d);     // graph replays add the kernels they run
#define KDSS_LAUNCH_CHECK() \
    (::kdss::count_launch(), ::kdss::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__))

// Device error word bits set by kernels (never a trap).
enum : int {
    DERR_NONE = 0,
    DERR_BAD_ID = 1,        // an id outside [0, n)
    DERR_OVERFLOW = 2,      // a count left its exact range
    DERR_TIMEOUT = 4,       // a bounded wait expired
    DERR_CAPACITY = 8,      // a bounded buffer would overflow (skipped)
    DERR_LOGIC = 16,        // an invariant failed (e.g. water-filling found no room)
};

// ---------------------------------------------------------------------------
// Device memory through the caller's allocator or stream-ordered cudaMalloc.
// ---------------------------------------------------------------------------
struct Ctx {
    cudaStream_t stream = nullptr;
    kdss_alloc_fn alloc = nullptr;
    kdss_free_fn free = nullptr;
    void *actx = nullptr;
    int num_sms = 0;
    int device = 0;
    uint32_t flags = 0;   // kdss_opts.flags of the call
};

Ctx make_ctx(const kdss_opts *o);
void *dalloc(const Ctx &c, size_t bytes);
void dfree(const Ctx &c, void *p, size_t bytes);

template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    Ctx ctx{};
    DBuf() = default;
    DBuf(const Ctx &c, size_t count) : n(count), ctx(c) {
        p = count ? static_cast<T *>(dalloc(c, count * sizeof(T))) : nullptr;
    }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), ctx(o.ctx) { o.p = nullptr; o.n = 0; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) { reset(); p = o.p; n = o.n; ctx = o.ctx; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DBuf() { reset(); }
    void reset() {
        if (p) dfree(ctx, p, n * sizeof(T));
        p = nullptr; n = 0;
    }
    T *get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// Pinned-free host <-> device helpers on the context stream (synchronous).
template <class T>
void to_host(const Ctx &c, T *dst, const T *src, size_t count) {
    if (!count) return;
    KDSS_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDeviceToHost, c.stream));
    KDSS_CUDA(cudaStreamSynchronize(c.stream));
}
template <class T>
void to_device(const Ctx &c, T *dst, const T *src, size_t count) {
    if (!count) return;
    KDSS_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, c.stream));
}
void sync(const Ctx &c);
void zero(const Ctx &c, void *p, size_t bytes);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Unsigned 128-bit integer for clique counts beyond 64 bits (Lemma 2.6 counts
// C(p, k - h) of long pairs, c_k and the prefix counts of the extraction).
// Trivially default-constructible so that it can live in shared memory.
struct U128 {
    unsigned long long lo, hi;
    U128() = default;
    __host__ __device__ constexpr U128(int v)
        : lo((unsigned long long)(long long)v), hi(v < 0 ? ~0ull : 0ull) {}
    __host__ __device__ constexpr U128(unsigned long long l, unsigned long long h) : lo(l), hi(h) {}
};
__host__ __device__ inline U128 operator+(U128 a, U128 b) {
    U128 r(a.lo + b.lo, a.hi + b.hi);
    if (r.lo < a.lo) ++r.hi;
    return r;
}
__host__ __device__ inline U128 operator-(U128 a, U128 b) {
    U128 r(a.lo - b.lo, a.hi - b.hi);
    if (a.lo < b.lo) --r.hi;
    return r;
}
__host__ __device__ inline U128 &operator+=(U128 &a, U128 b) { a = a + b; return a; }
__host__ __device__ inline bool operator==(U128 a, U128 b) { return a.lo == b.lo && a.hi == b.hi; }
__host__ __device__ inline bool operator!=(U128 a, U128 b) { return !(a == b); }
// marker of a binomial that needs more than 128 bits
constexpr U128 U128_OVF(~0ull, ~0ull);
inline int bit_length_u128(U128 x) {
    int b = 0;
    unsigned long long h = x.hi, l = x.lo;
    if (h) { b = 64; l = h; }
    while (l) { ++b; l >>= 1; }
    return b;
}
inline double u128_to_double(U128 x) { return (double)x.hi * 18446744073709551616.0 + (double)x.lo; }
inline int bit_length(uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return b; }

// Grid size for a grid-stride kernel: a multiple of the SM count.
int grid_for(const Ctx &c, int64_t work_items, int block, int blocks_per_sm = 8);

// ---------------------------------------------------------------------------
// Primitives (scan_sort.cu)
// ---------------------------------------------------------------------------
// out[i] = sum of in[0..i) for i < n; returns the total (synchronises).
int64_t exclusive_scan_i64(const Ctx &c, const int64_t *in, int64_t *out, int64_t n);
// In-place variant that does not read the total back (stream-ordered).
void exclusive_scan_i64_async(const Ctx &c, const int64_t *in, int64_t *out, int64_t n);
void inclusive_scan_u64_async(const Ctx &c, const uint64_t *in, uint64_t *out, int64_t n);
void inclusive_scan_u128_async(const Ctx &c, const U128 *in, U128 *out, int64_t n);

// Stable LSD radix sort of 64-bit keys (with optional int32 payload) on the
// digit positions that cover bits [lo, hi) of each range in `ranges`.
// keys/vals are sorted in place (double-buffered internally).
struct BitRange { int lo, hi; };
void radix_sort_u64(const Ctx &c, uint64_t *keys, int32_t *vals, int64_t n,
                    const std::vector<BitRange> &ranges);

// Offsets of a sorted key array whose high 32 bits are a row index:
// off[r] = first position with row >= r, r = 0..nrows.
void row_offsets_from_sorted(const Ctx &c, const uint64_t *keys, int64_t nkeys, int64_t nrows,
                             int64_t *off);

// Max of a u64 array (synchronises).
uint64_t reduce_max_u64(const Ctx &c, const uint64_t *in, int64_t n);

// State of the bounded grid barrier of the cooperative kernels
// (grid_sync_count below): arrivals so far, cleared by the host before each
// launch.  Every wait gives up after a deadline (ns of %globaltimer) and sets
// DERR_TIMEOUT in the kernel's error word.
struct GridBarrier {
    unsigned int count;
};

}  // namespace kdss

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
namespace kdss {

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier on a counter that only grows: every block adds 1 per barrier,
// and barrier number e (from 1) is passed once the counter reaches e x the
// number of blocks.  The counter starts at zero for each launch (the host
// clears it), so no block resets anything: an arrival is one release add and
// a wait polls with acquire loads.  Returns false when the wait timed out
// (the error word then holds DERR_TIMEOUT).
__device__ __forceinline__ bool grid_sync_count(unsigned int *count, unsigned int target, int *err,
                                                uint64_t timeout_ns) {
    __syncthreads();
    __shared__ int s_okc;
    if (threadIdx.x == 0) {
        // the release orders every write of the block before the arrival:
        // bar.sync above places the other threads' writes before it
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
        int ok = 1;
        const uint64_t t0 = globaltimer_ns();
        unsigned int polls = 0;
        while (true) {
            unsigned int cur;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(count) : "memory");
            if ((int)(cur - target) >= 0) break;
            if ((++polls & 255u) == 0u && globaltimer_ns() - t0 > timeout_ns) {
                atomicOr(err, DERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        s_okc = ok;
    }
    __syncthreads();
    return s_okc != 0;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace kdss
#endif
