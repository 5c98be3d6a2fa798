// noalloc.cu -- Frank-Wolfe iterations that allocate no device memory.
//
// Some callers cannot allocate device memory while they run the solver: a
// process whose device memory is reserved up front and handed out by its own
// arena (so a cudaMalloc behind its back could fail or break its budget), a
// serving loop that must keep a fixed footprint, or code that must not
// perform an implicitly synchronising allocation in the middle of its GPU
// work.  kdss_fw_iterate_noalloc serves them: the caller owns r, the SCT was
// built beforehand, and the scratch the iterations need lives in one
// file-scope device array of fixed size that every GPU loading this library
// holds until the process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "handles.cuh"

namespace {

using namespace kdss;

// The scratch of all allocation-free calls.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_addr[MAX_DEVICES] = {};
void *g_addr_ctx[MAX_DEVICES] = {};  // the context each cached address belongs to

// The calling thread's current CUDA context (the driver's cuCtxGetCurrent,
// reached through the runtime's entry-point query so that the library needs
// no link against the driver library); nullptr when it cannot be queried.
void *current_context() {
    using fn_t = int (*)(void **);
    static fn_t fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (fn_t) nullptr;
        }
        return reinterpret_cast<fn_t>(f);
    }();
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

// Device address of the scratch array on `dev` (the current device).  In host
// code the array's name stands for a host-side shadow, not device memory, so
// the address is looked up once per device and context and cached; a new
// context on the device (after cudaDeviceReset) triggers a new lookup.
void *scratch_address(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= MAX_DEVICES) fail(KDSS_ERR_UNSUPPORTED, "device index out of range");
    void *ctx = current_context();
    if (!g_addr[dev] || g_addr_ctx[dev] != ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(KDSS_ERR_CUDA, std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                                    cudaGetErrorString(e));
        }
        g_addr[dev] = p;
        g_addr_ctx[dev] = ctx;
    }
    return g_addr[dev];
}

// r must be device (or managed) memory of `dev` from its first to its last
// element; a host pointer or another device's memory would make the kernels
// fault or write where they must not.
void check_r_on_device(const uint64_t *r, int64_t n, int dev) {
    if (n <= 0) return;
    for (const uint64_t *p : {r, r + (n - 1)}) {
        cudaPointerAttributes a{};
        const cudaError_t e = cudaPointerGetAttributes(&a, p);
        if (e != cudaSuccess) {
            cudaGetLastError();
            fail(KDSS_ERR_INVALID_ARG, std::string("r: cudaPointerGetAttributes failed: ") +
                                           cudaGetErrorString(e));
        }
        const bool dev_mem = a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
        if (!dev_mem || a.device != dev) {
            char buf[200];
            snprintf(buf, sizeof buf,
                     "r must be device memory of device %d holding n = %lld uint64 values "
                     "(element %s is %s)", dev, (long long)n, p == r ? "0" : "n - 1",
                     dev_mem ? "on another device" : "not device memory");
            fail(KDSS_ERR_INVALID_ARG, buf);
        }
    }
}

inline size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

namespace kdss {
void set_last_error(const std::string &msg);  // api.cu: the text kdss_last_error() returns
}

extern "C" kdss_status kdss_fw_iterate_noalloc(const kdss_sct *s, uint64_t *r, int32_t t_done,
                                               int32_t T, void *stream) {
    try {
        if (!s || !r) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
        if (s->kmax_multi) fail(KDSS_ERR_INVALID_ARG, "a k-agnostic SCT: restrict it to one k first");
        if (s->shared) fail(KDSS_ERR_INVALID_ARG, "a prefix-shared SCT: iterate it with kdss_fw_iterate");
        if (T < 0 || t_done < 0) fail(KDSS_ERR_INVALID_ARG, "T and t_done must be >= 0");
        const SctDev &sd = s->s;
        int dev = 0;
        KDSS_CUDA(cudaGetDevice(&dev));
        if (dev != s->ctx.device)
            fail(KDSS_ERR_INVALID_ARG, "the SCT lives on another device than the current one");
        check_r_on_device(r, sd.n, dev);
        // exactness of the cumulative r: r_t(u) <= t * c_k
        const long double ck = (long double)sd.ck_lo + (long double)sd.ck_hi * 18446744073709551616.0L;
        if ((long double)((int64_t)t_done + T) * ck >= 9.2e18L)
            fail(KDSS_ERR_OVERFLOW, "(t_done + T) * c_k leaves the exact range of r");
        // scratch layout: counters | delta [n] | slow-pair list [short pairs]
        const int64_t short_pairs = sd.class_begin[3] - sd.class_begin[0];
        int num_sms = 0;
        KDSS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
        const size_t off_acc = 256;
        const size_t off_slow = off_acc + round_up((size_t)sd.n * sizeof(uint64_t));
        const size_t need =
            off_slow + round_up((size_t)slow_list_capacity(short_pairs, num_sms) * sizeof(int32_t));
        if (need > NOALLOC_SCRATCH_BYTES) {
            char buf[256];
            snprintf(buf, sizeof buf,
                     "the allocation-free FW entry point holds at most %zu bytes of scratch; "
                     "n = %lld nodes and %lld short pairs need %zu",
                     NOALLOC_SCRATCH_BYTES, (long long)sd.n, (long long)short_pairs, need);
            fail(KDSS_ERR_INVALID_ARG, buf);
        }
        Ctx c;
        c.stream = static_cast<cudaStream_t>(stream);
        c.device = dev;
        c.num_sms = num_sms;
        unsigned char *base = static_cast<unsigned char *>(scratch_address(dev));
        int *slow_count = reinterpret_cast<int *>(base);
        int *err = reinterpret_cast<int *>(base + 4);
        unsigned long long *maxr = reinterpret_cast<unsigned long long *>(base + 8);
        uint64_t *acc = reinterpret_cast<uint64_t *>(base + off_acc);
        int32_t *slow = reinterpret_cast<int32_t *>(base + off_slow);
        // the array keeps the previous call's contents: clear what must start at zero
        KDSS_CUDA(cudaMemsetAsync(base, 0, off_acc, c.stream));
        if (sd.n > 0) KDSS_CUDA(cudaMemsetAsync(acc, 0, (size_t)sd.n * sizeof(uint64_t), c.stream));
        fw_run_external(c, sd, r, acc, slow, slow_count, err, maxr, T);
        int herr = 0;
        KDSS_CUDA(cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, c.stream));
        KDSS_CUDA(cudaStreamSynchronize(c.stream));
        if (herr) fail(KDSS_ERR_CUDA, "FW iteration: water-filling invariant failed on the device");
    } catch (const Error &e) {
        kdss::set_last_error(e.msg);
        return e.code;
    } catch (...) {
        kdss::set_last_error("unknown internal error");
        return KDSS_ERR_CUDA;
    }
    kdss::set_last_error("");
    return KDSS_OK;
}
