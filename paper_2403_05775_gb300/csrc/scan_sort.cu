// scan_sort.cu -- device-wide scans, a stable LSD radix sort and small
// reductions used by the graph build and the extraction.
#include "kdss_internal.cuh"

namespace kdss {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ T shfl_up_any(T v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
template <>
__device__ __forceinline__ U128 shfl_up_any<U128>(U128 v, int o) {
    return U128(__shfl_up_sync(0xffffffffu, v.lo, o), __shfl_up_sync(0xffffffffu, v.hi, o));
}

template <class T>
__device__ __forceinline__ T warp_inclusive(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = shfl_up_any(v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of one value per thread over the block; *total (shared
// memory) receives the block sum.
template <class T>
__device__ __forceinline__ T block_exclusive(T v, T *total) {
    constexpr int NW = SCAN_THREADS / 32;
    __shared__ T s_w[NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_inclusive(v);
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        T x = lane < NW ? s_w[lane] : T(0);
        T xi = warp_inclusive(x);
        if (lane < NW) s_w[lane] = xi - x;
        if (lane == NW - 1) *total = xi;
    }
    __syncthreads();
    return s_w[w] + inc - v;
}

template <class T>
__global__ void k_tile_sums(const T *in, int64_t n, T *sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T acc = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        if (j < n) acc += in[j];
    }
    __shared__ T s_total;
    block_exclusive<T>(acc, &s_total);
    __syncthreads();
    if (threadIdx.x == 0) sums[blockIdx.x] = s_total;
}

template <class T, bool INCLUSIVE>
__global__ void k_tile_scan(const T *in, T *out, int64_t n, const T *offsets) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T v[SCAN_ITEMS];
    T acc = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        v[i] = j < n ? in[j] : T(0);
        acc += v[i];
    }
    __shared__ T s_total;
    T run = block_exclusive<T>(acc, &s_total) + (offsets ? offsets[blockIdx.x] : T(0));
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t j = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        T x = v[i];
        if (INCLUSIVE) run += x;
        if (j < n) out[j] = run;
        if (!INCLUSIVE) run += x;
    }
}

template <class T, bool INCLUSIVE>
void scan_impl(const Ctx &c, const T *in, T *out, int64_t n) {
    if (n <= 0) return;
    int64_t nb = ceil_div(n, SCAN_TILE);
    if (nb == 1) {
        k_tile_scan<T, INCLUSIVE><<<1, SCAN_THREADS, 0, c.stream>>>(in, out, n, nullptr);
        KDSS_LAUNCH_CHECK();
        return;
    }
    DBuf<T> sums(c, (size_t)nb), offs(c, (size_t)nb);
    k_tile_sums<T><<<(unsigned)nb, SCAN_THREADS, 0, c.stream>>>(in, n, sums.p);
    KDSS_LAUNCH_CHECK();
    scan_impl<T, false>(c, sums.p, offs.p, nb);
    k_tile_scan<T, INCLUSIVE><<<(unsigned)nb, SCAN_THREADS, 0, c.stream>>>(in, out, n, offs.p);
    KDSS_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------
// A block sorts a tile of `rounds` x 256 keys, 256 per round.  The rounds
// per tile grow with n so that the grid stays at about two blocks per SM: a
// small sort (1e5 keys) then takes one or two short rounds per block instead
// of a few blocks walking 32 rounds each.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_MAX_ROUNDS = 32;

__global__ void k_rs_hist(const uint64_t *keys, int64_t n, int shift, uint32_t mask,
                          int32_t *hist, int64_t nblocks, int rounds) {
    __shared__ int32_t cnt[RS_WARPS][256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const int64_t tile = (int64_t)RS_THREADS * rounds;
    int64_t base = (int64_t)blockIdx.x * tile;
    int64_t end = base + tile < n ? base + tile : n;
    for (int64_t i = base + threadIdx.x; i < end; i += RS_THREADS) {
        uint32_t d = (uint32_t)(keys[i] >> shift) & mask;
        atomicAdd(&cnt[w][d], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        int32_t s = 0;
#pragma unroll
        for (int q = 0; q < RS_WARPS; ++q) s += cnt[q][d];
        hist[(int64_t)d * nblocks + blockIdx.x] = s;
    }
}

__global__ void k_rs_scatter(const uint64_t *kin, const int32_t *vin, uint64_t *kout,
                             int32_t *vout, int64_t n, int shift, uint32_t mask,
                             const int32_t *hist_scan, int64_t nblocks, int rounds) {
    __shared__ int32_t s_base[256];
    __shared__ int32_t s_run[256];
    __shared__ int32_t s_w[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) {
        s_base[d] = hist_scan[(int64_t)d * nblocks + blockIdx.x];
        s_run[d] = 0;
    }
    int64_t tile = (int64_t)blockIdx.x * RS_THREADS * rounds;
    for (int r = 0; r < rounds; ++r) {
        int64_t i = tile + (int64_t)r * RS_THREADS + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0ull;
        int d = valid ? (int)((uint32_t)(key >> shift) & mask) : 256;
        for (int q = threadIdx.x; q < RS_WARPS * 256; q += RS_THREADS) (&s_w[0][0])[q] = 0;
        __syncthreads();
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) s_w[w][d] = __popc(peers);
        __syncthreads();
        {
            int t = threadIdx.x;  // one digit per thread (256 threads)
            int32_t run = s_run[t];
#pragma unroll
            for (int q = 0; q < RS_WARPS; ++q) {
                int32_t cq = s_w[q][t];
                s_w[q][t] = run;
                run += cq;
            }
            s_run[t] = run;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = (int64_t)s_base[d] + s_w[w][d] + rank;
            kout[pos] = key;
            if (vin) vout[pos] = vin[i];
        }
        __syncthreads();
        if (tile + (int64_t)(r + 1) * RS_THREADS >= n) break;  // uniform over the block
    }
    (void)lane;
}

__global__ void k_row_offsets(const uint64_t *keys, int64_t nk, int64_t nrows, int64_t *off) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= nk;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = i < nk ? (int64_t)(keys[i] >> 32) : nrows;
        int64_t prev = i > 0 ? (int64_t)(keys[i - 1] >> 32) : -1;
        if (row > nrows) row = nrows;
        for (int64_t r = prev + 1; r <= row; ++r) off[r] = i;
    }
}

__global__ void k_max_u64(const uint64_t *in, int64_t n, unsigned long long *out) {
    uint64_t m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = in[i] > m ? in[i] : m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)m);
}

}  // namespace

int64_t exclusive_scan_i64(const Ctx &c, const int64_t *in, int64_t *out, int64_t n) {
    if (n <= 0) return 0;
    scan_impl<int64_t, false>(c, in, out, n);
    int64_t last_in = 0, last_out = 0;
    KDSS_CUDA(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
    KDSS_CUDA(cudaMemcpyAsync(&last_out, out + n - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    return last_in + last_out;
}

void exclusive_scan_i64_async(const Ctx &c, const int64_t *in, int64_t *out, int64_t n) {
    scan_impl<int64_t, false>(c, in, out, n);
}

void inclusive_scan_u64_async(const Ctx &c, const uint64_t *in, uint64_t *out, int64_t n) {
    scan_impl<uint64_t, true>(c, in, out, n);
}

void inclusive_scan_u128_async(const Ctx &c, const U128 *in, U128 *out, int64_t n) {
    scan_impl<U128, true>(c, in, out, n);
}

void radix_sort_u64(const Ctx &c, uint64_t *keys, int32_t *vals, int64_t n,
                    const std::vector<BitRange> &ranges) {
    if (n <= 1) return;
    if (n > (int64_t)INT32_MAX) fail(KDSS_ERR_UNSUPPORTED, "radix sort of more than 2^31 keys");
    struct Pass { int shift; uint32_t mask; };
    std::vector<Pass> passes;
    for (const BitRange &r : ranges)
        for (int s = r.lo; s < r.hi; s += 8) {
            int bits = r.hi - s < 8 ? r.hi - s : 8;
            passes.push_back({s, (1u << bits) - 1u});
        }
    if (passes.empty()) return;
    const int rounds = (int)std::min<int64_t>(
        RS_MAX_ROUNDS, std::max<int64_t>(1, ceil_div(n, (int64_t)RS_THREADS * 2 * c.num_sms)));
    int64_t nb = ceil_div(n, (int64_t)RS_THREADS * rounds);
    DBuf<uint64_t> kalt(c, (size_t)n);
    DBuf<int32_t> valt(c, vals ? (size_t)n : 0);
    DBuf<int32_t> hist(c, (size_t)(256 * nb)), hscan(c, (size_t)(256 * nb));
    uint64_t *ka = keys, *kb = kalt.p;
    int32_t *va = vals, *vb = valt.p;
    for (const Pass &p : passes) {
        k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, c.stream>>>(ka, n, p.shift, p.mask, hist.p, nb,
                                                            rounds);
        KDSS_LAUNCH_CHECK();
        scan_impl<int32_t, false>(c, hist.p, hscan.p, 256 * nb);
        k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, c.stream>>>(ka, va, kb, vb, n, p.shift, p.mask,
                                                                hscan.p, nb, rounds);
        KDSS_LAUNCH_CHECK();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        KDSS_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                                  c.stream));
        if (vals)
            KDSS_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * sizeof(int32_t),
                                      cudaMemcpyDeviceToDevice, c.stream));
    }
}

void row_offsets_from_sorted(const Ctx &c, const uint64_t *keys, int64_t nkeys, int64_t nrows,
                             int64_t *off) {
    int block = 256;
    int grid = grid_for(c, nkeys + 1, block);
    k_row_offsets<<<grid, block, 0, c.stream>>>(keys, nkeys, nrows, off);
    KDSS_LAUNCH_CHECK();
}

uint64_t reduce_max_u64(const Ctx &c, const uint64_t *in, int64_t n) {
    DBuf<unsigned long long> out(c, 1);
    zero(c, out.p, sizeof(unsigned long long));
    if (n > 0) {
        int block = 256;
        k_max_u64<<<grid_for(c, n, block), block, 0, c.stream>>>(in, n, out.p);
        KDSS_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    to_host(c, &h, out.p, 1);
    return h;
}

}  // namespace kdss
