// runtime.cu -- errors, device allocation and launch sizing for the solver.
#include <atomic>
#include <cstdarg>
#include <cstring>

#include "kdss_internal.cuh"

namespace kdss {

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;  // this thread's launches (graph capture counts)
void count_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}
long long launches() { return g_launches.load(std::memory_order_relaxed); }
long long thread_launches() { return t_launches; }
void add_launches(long long d) { g_launches.fetch_add(d, std::memory_order_relaxed); }

void fail(kdss_status code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear the sticky-free allocation error
        fail(KDSS_ERR_OOM, buf);
    }
    fail(KDSS_ERR_CUDA, buf);
}

void check_device_array(const void *p, size_t bytes, const char *what, int dev) {
    if (bytes == 0) return;
    if (dev < 0) KDSS_CUDA(cudaGetDevice(&dev));
    const char *ends[2] = {static_cast<const char *>(p), static_cast<const char *>(p) + (bytes - 1)};
    for (int i = 0; i < 2; ++i) {
        cudaPointerAttributes a{};
        const cudaError_t e = cudaPointerGetAttributes(&a, ends[i]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            char buf[256];
            snprintf(buf, sizeof buf, "%s: cudaPointerGetAttributes failed: %s", what,
                     cudaGetErrorString(e));
            fail(KDSS_ERR_INVALID_ARG, buf);
        }
        const bool dev_mem = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
        if (!dev_mem || a.device != dev) {
            char buf[256];
            snprintf(buf, sizeof buf,
                     "%s must be device memory of device %d over its %zu bytes (its %s byte is %s)",
                     what, dev, bytes, i ? "last" : "first",
                     dev_mem ? "on another device" : "not device memory");
            fail(KDSS_ERR_INVALID_ARG, buf);
        }
    }
}

Ctx make_ctx(const kdss_opts *o) {
    Ctx c;
    if (o) {
        c.stream = static_cast<cudaStream_t>(o->stream);
        c.alloc = o->alloc;
        c.free = o->free;
        c.actx = o->alloc_ctx;
        c.flags = o->flags;
        if ((c.alloc == nullptr) != (c.free == nullptr))
            fail(KDSS_ERR_INVALID_ARG, "opts.alloc and opts.free must be set together");
        if (o->rule < KDSS_RULE_DEFAULT || o->rule > KDSS_RULE_CONTINUOUS)
            fail(KDSS_ERR_INVALID_ARG, "unknown rule");
        if (o->rule == KDSS_RULE_INTEGER && o->precision == KDSS_FP32K)
            fail(KDSS_ERR_UNSUPPORTED, "KDSS_FP32K runs the continuous rule; the integer rule of "
                                       "Alg. 3 is held in KDSS_INT64 or KDSS_FP64");
        if (o->rule == KDSS_RULE_CONTINUOUS && o->precision != KDSS_FP32K)
            fail(KDSS_ERR_UNSUPPORTED, "the continuous rule runs in KDSS_FP32K; KDSS_INT64 and "
                                       "KDSS_FP64 hold the integer rule of Alg. 3");
    }
    KDSS_CUDA(cudaGetDevice(&c.device));
    KDSS_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device));
    if (!c.alloc) {
        // Without a caller allocator the library draws from the device's
        // stream-ordered pool; let the pool keep freed memory for reuse
        // instead of returning it at every synchronisation (a setting of this
        // process's pool only).
        static thread_local int tuned_device = -1;
        if (tuned_device != c.device) {
            cudaMemPool_t pool;
            if (cudaDeviceGetDefaultMemPool(&pool, c.device) == cudaSuccess) {
                uint64_t keep = ~0ull;
                cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            }
            cudaGetLastError();
            tuned_device = c.device;
        }
    }
    return c;
}

void *dalloc(const Ctx &c, size_t bytes) {
    if (bytes == 0) return nullptr;
    void *p = nullptr;
    if (c.alloc) {
        p = c.alloc(bytes, c.stream, c.actx);
        if (!p) {
            char buf[128];
            snprintf(buf, sizeof buf, "device allocation of %zu bytes failed", bytes);
            fail(KDSS_ERR_OOM, buf);
        }
        return p;
    }
    cudaError_t e = cudaMallocAsync(&p, bytes, c.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "cudaMallocAsync of %zu bytes failed: %s", bytes,
                 cudaGetErrorString(e));
        fail(e == cudaErrorMemoryAllocation ? KDSS_ERR_OOM : KDSS_ERR_CUDA, buf);
    }
    return p;
}

void dfree(const Ctx &c, void *p, size_t bytes) {
    if (!p) return;
    if (c.free) {
        c.free(p, bytes, c.stream, c.actx);
        return;
    }
    cudaFreeAsync(p, c.stream);  // destructors must not throw
}

void sync(const Ctx &c) { KDSS_CUDA(cudaStreamSynchronize(c.stream)); }

void zero(const Ctx &c, void *p, size_t bytes) {
    if (bytes) KDSS_CUDA(cudaMemsetAsync(p, 0, bytes, c.stream));
}

int grid_for(const Ctx &c, int64_t work_items, int block, int blocks_per_sm) {
    int64_t need = ceil_div(work_items > 0 ? work_items : 1, block);
    int64_t cap = (int64_t)c.num_sms * blocks_per_sm;
    if (need >= cap) return (int)cap;
    return (int)need;
}

}  // namespace kdss
