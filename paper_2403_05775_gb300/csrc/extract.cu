// extract.cu -- step A6: the densest prefix of the nodes sorted by r (the
// final sort and prefix step of Alg. 2).
//
// 1. Sort V by r non-increasing, ties by ascending id: a stable LSD radix sort
//    of key = max(r) - r over ids 0..n-1 (key bits of the float / double
//    representation for the floating-point states).
// 2. |C_k(V_i)| for every prefix length i from the pairs: by Lemmas 2.5-2.6 a
//    pair holds C(#{V_p nodes in V_i}, k - h) k-cliques of V_i once V_h is
//    inside V_i.  With mh the last position of a V_h node, the pair adds
//    C(c0, k - h) at prefix length mh + 1 (c0 = V_p nodes before mh), and for
//    each later V_p node at position q the increment
//    C(c + 1, k - h) - C(c, k - h) = C(c, k - h - 1) at length q + 1
//    (c = V_p nodes before q).  A scan of the increments gives C_k(V_i).
//    The same pass adds n_C at the length where the whole pair is inside,
//    whose scan is sum_{P inside V_i} n_C = i * rho'(V_i) (Thm 3.6).
// 3. i* = the largest i maximising C_k(V_i) / i, compared exactly by
//    128-bit cross-multiplication.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "fw.cuh"

namespace kdss {

void extract_prefix(const Ctx &c, const SctDev &s, const StateDev &st, kdss_result *out);

namespace {

constexpr unsigned FULL = 0xffffffffu;

__global__ void k_keys_u64(int64_t n, const uint64_t *r, uint64_t maxv, uint64_t *keys,
                           int32_t *vals) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        keys[v] = maxv - r[v];
        vals[v] = (int32_t)v;
    }
}
// FP64 storage: the integer value of each r, so that the key has only as
// many bits as max r (the raw bit patterns would need all 64).
__global__ void k_keys_f64(int64_t n, const uint64_t *r, uint64_t maxv, uint64_t *keys,
                           int32_t *vals) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        keys[v] = maxv - (uint64_t)__longlong_as_double((long long)r[v]);
        vals[v] = (int32_t)v;
    }
}
__global__ void k_keys_f32(int64_t n, const float *r, uint32_t maxbits, uint64_t *keys,
                           int32_t *vals) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        float x = r[v];
        uint32_t b = x > 0.f ? (uint32_t)__float_as_int(x) : 0u;
        keys[v] = (uint64_t)(maxbits - b);
        vals[v] = (int32_t)v;
    }
}
__global__ void k_max_f32bits(int64_t n, const float *r, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        float x = r[v];
        unsigned long long b = x > 0.f ? (unsigned long long)(uint32_t)__float_as_int(x) : 0ull;
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(FULL, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void k_positions(int64_t n, const int32_t *order, int32_t *pos) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        pos[order[i]] = (int32_t)i;
}

template <int G>
__device__ __forceinline__ int gmax_i32(int v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
template <int G>
__device__ __forceinline__ int gsum_i32(int v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Prefix-count increments of the pairs [b, e): a group of G lanes per pair.
// 128-bit atomic add: the carry of each low-word add goes to the high word,
// so concurrent adds sum exactly.
__device__ __forceinline__ void atomic_add_u128(U128 *a, U128 x) {
    if (x.lo == 0 && x.hi == 0) return;
    const unsigned long long old = atomicAdd(&a->lo, x.lo);
    const unsigned long long carry = (old + x.lo < old) ? 1ull : 0ull;
    if (x.hi + carry) atomicAdd(&a->hi, x.hi + carry);
}

// Counts of the narrow form (every count below 2^64: 64-bit table and
// histograms) or the wide form (128-bit).
template <bool WIDE>
struct EventTables {
    const uint64_t *binom;
    const U128 *binom128;
    unsigned long long *hist, *fhist;
    U128 *hist128, *fhist128;
    __device__ __forceinline__ void add(bool full, int row, int bcols, int col, int at) const {
        if constexpr (WIDE) {
            atomic_add_u128((full ? fhist128 : hist128) + at, binom128[(size_t)row * bcols + col]);
        } else {
            const uint64_t v = __ldg(binom + (size_t)row * bcols + col);
            if (v) atomicAdd((full ? fhist : hist) + at, (unsigned long long)v);
        }
    }
};

template <int G, int NPL, bool WIDE>
__global__ void __launch_bounds__(256)
k_prefix_events(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
                const uint8_t *__restrict__ hcnt, int64_t b, int64_t e,
                const int32_t *__restrict__ pos, EventTables<WIDE> tb, int bcols, int k) {
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t np = e - b;
    for (int64_t wb = warp * GPW; wb < np; wb += nwarps * GPW) {
        const int64_t qi = wb + lane / G;
        const bool active = qi < np;
        const int64_t q = b + qi;
        int64_t off0 = 0;
        int len = 0, h = 0;
        if (active) {
            off0 = pair_off[q];
            len = (int)(pair_off[q + 1] - off0);
            h = hcnt[q];
        }
        // pairs outside P_k (a k-agnostic SCT extracted at k) hold no k-clique
        const bool inpk = active && h <= k && k <= len;
        const int p = len - h;
        int ps[NPL];
        bool hold[NPL], valid[NPL];
        int mh = -1, mall = -1;
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int j = s * G + gl;
            valid[s] = inpk && j < len;
            const int32_t raw = valid[s] ? __ldg(nodes + off0 + j) : 0;
            hold[s] = raw < 0;
            ps[s] = valid[s] ? __ldg(pos + (raw & 0x7fffffff)) : -1;
            if (valid[s] && hold[s]) mh = max(mh, ps[s]);
            if (valid[s]) mall = max(mall, ps[s]);
        }
        mh = gmax_i32<G>(mh);
        mall = gmax_i32<G>(mall);
        // c0 = pivot nodes before the last hold node
        int c0 = 0;
#pragma unroll
        for (int s = 0; s < NPL; ++s)
            if (valid[s] && !hold[s] && ps[s] < mh) ++c0;
        c0 = gsum_i32<G>(c0);
        // rank of each later pivot node among the pivot positions
        int rk[NPL];
#pragma unroll
        for (int s = 0; s < NPL; ++s) rk[s] = 0;
        for (int s2 = 0; s2 < NPL; ++s2) {
            for (int l2 = 0; l2 < G; ++l2) {
                const int pv = __shfl_sync(FULL, (valid[s2] && !hold[s2]) ? ps[s2] : -1, gbase + l2);
#pragma unroll
                for (int s = 0; s < NPL; ++s)
                    if (pv >= 0 && pv < ps[s]) ++rk[s];
            }
        }
        if (inpk) {
            const int kh = k - h;
            if (gl == 0) {
                tb.add(false, c0, bcols, kh, mh + 1);     // C(c0, k - h) once V_h is inside
                tb.add(true, p, bcols, kh, mall + 1);     // n_C once the whole pair is inside
            }
            if (kh >= 1) {
#pragma unroll
                for (int s = 0; s < NPL; ++s)
                    if (valid[s] && !hold[s] && ps[s] > mh) tb.add(false, rk[s], bcols, kh - 1, ps[s] + 1);
            }
        }
    }
}

// a / i > b / j, exact (a, b < 2^64, i, j < 2^63)
__device__ __forceinline__ int frac_cmp(unsigned long long a, unsigned long long i,
                                        unsigned long long b, unsigned long long j) {
    unsigned long long ahi = __umul64hi(a, j), alo = a * j;
    unsigned long long bhi = __umul64hi(b, i), blo = b * i;
    if (ahi != bhi) return ahi > bhi ? 1 : -1;
    if (alo != blo) return alo > blo ? 1 : -1;
    return 0;
}
// the same for 128-bit counts (i, j < 2^63): 192-bit cross products
__device__ __forceinline__ void mul_u128_u64(U128 a, unsigned long long j, unsigned long long &w2,
                                             unsigned long long &w1, unsigned long long &w0) {
    w0 = a.lo * j;
    const unsigned long long c0 = __umul64hi(a.lo, j);
    const unsigned long long t = a.hi * j;
    w1 = t + c0;
    w2 = __umul64hi(a.hi, j) + (w1 < t ? 1ull : 0ull);
}
__device__ __forceinline__ int frac_cmp(U128 a, unsigned long long i, U128 b, unsigned long long j) {
    unsigned long long a2, a1, a0, b2, b1, b0;
    mul_u128_u64(a, j, a2, a1, a0);
    mul_u128_u64(b, i, b2, b1, b0);
    if (a2 != b2) return a2 > b2 ? 1 : -1;
    if (a1 != b1) return a1 > b1 ? 1 : -1;
    if (a0 != b0) return a0 > b0 ? 1 : -1;
    return 0;
}
__device__ __forceinline__ unsigned long long shfl_xor_ct(unsigned long long v, int o) {
    return __shfl_xor_sync(FULL, v, o);
}
__device__ __forceinline__ U128 shfl_xor_ct(U128 v, int o) {
    return U128(__shfl_xor_sync(FULL, v.lo, o), __shfl_xor_sync(FULL, v.hi, o));
}

// Best prefix of a scanned count array: largest ratio, ties to the larger i.
template <class CT>
__device__ __forceinline__ void better(CT &a, long long &i, CT b, long long j) {
    if (j <= 0) return;
    if (i <= 0) { a = b; i = j; return; }
    int c = frac_cmp(b, (unsigned long long)j, a, (unsigned long long)i);
    if (c > 0 || (c == 0 && j > i)) { a = b; i = j; }
}

template <class CT>
__device__ __forceinline__ void block_best(CT &a, long long &i, CT *sa, long long *si) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        CT b = shfl_xor_ct(a, o);
        long long j = __shfl_xor_sync(FULL, i, o);
        better(a, i, b, j);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sa[w] = a; si[w] = i; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? sa[lane] : CT(0);
        i = lane < nw ? si[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            CT b = shfl_xor_ct(a, o);
            long long j = __shfl_xor_sync(FULL, i, o);
            better(a, i, b, j);
        }
    }
}

template <class CT>
__global__ void k_argmax_partial(int64_t n, const CT *cnt, CT *pa, long long *pi) {
    CT a = CT(0);
    long long i = 0;
    for (int64_t x = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x <= n;
         x += (int64_t)gridDim.x * blockDim.x)
        better(a, i, cnt[x], x);
    __shared__ CT sa[32];
    __shared__ long long si[32];
    block_best(a, i, sa, si);
    if (threadIdx.x == 0) { pa[blockIdx.x] = a; pi[blockIdx.x] = i; }
}

template <class CT>
__global__ void k_argmax_final(int nb, const CT *pa, const long long *pi, CT *oa, long long *oi) {
    CT a = CT(0);
    long long i = 0;
    for (int x = threadIdx.x; x < nb; x += blockDim.x) better(a, i, pa[x], pi[x]);
    __shared__ CT sa[32];
    __shared__ long long si[32];
    block_best(a, i, sa, si);
    if (threadIdx.x == 0) { *oa = a; *oi = i; }
}

template <class CT>
void best_prefix(const Ctx &c, int64_t n, const CT *cnt, CT *a, long long *i) {
    const int B = 256;
    const int nb = std::min(grid_for(c, n, B, 4), 1024);
    DBuf<CT> pa(c, (size_t)nb), oa(c, 1);
    DBuf<long long> pi(c, (size_t)nb), oi(c, 1);
    k_argmax_partial<CT><<<nb, B, 0, c.stream>>>(n, cnt, pa.p, pi.p);
    KDSS_LAUNCH_CHECK();
    k_argmax_final<CT><<<1, 1024, 0, c.stream>>>(nb, pa.p, pi.p, oa.p, oi.p);
    KDSS_LAUNCH_CHECK();
    to_host(c, a, oa.p, 1);
    to_host(c, i, oi.p, 1);
}

template <int G, int NPL, bool WIDE>
void launch_events(const Ctx &c, const SctDev &s, int k, int cls, const int32_t *pos,
                   const EventTables<WIDE> &tb) {
    const int64_t b = s.class_begin[cls], e = s.class_begin[cls + 1];
    if (e <= b) return;
    const int64_t gpb = 8 * (32 / G);
    int grid = (int)std::min<int64_t>(ceil_div(e - b, gpb), (int64_t)c.num_sms * 16);
    k_prefix_events<G, NPL, WIDE><<<grid, 256, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, b, e,
                                                              pos, tb, s.bcols(), k);
    KDSS_LAUNCH_CHECK();
}

template <bool WIDE>
void launch_events_all(const Ctx &c, const SctDev &s, int k, const int32_t *pos,
                       const EventTables<WIDE> &tb) {
    launch_events<8, 1, WIDE>(c, s, k, 0, pos, tb);
    launch_events<8, 2, WIDE>(c, s, k, 1, pos, tb);
    launch_events<8, 4, WIDE>(c, s, k, 2, pos, tb);
    launch_events<32, 8, WIDE>(c, s, k, 3, pos, tb);
    launch_events<32, 32, WIDE>(c, s, k, 4, pos, tb);
}

}  // namespace

// The increments of every class, positions taken from pos (used by the
// segmented extraction of batches, whose positions index query segments).
void launch_prefix_events_all(const Ctx &c, const SctDev &s, const int32_t *pos,
                              unsigned long long *hist, unsigned long long *fhist) {
    EventTables<false> tb{s.binom.p, nullptr, hist, fhist, nullptr, nullptr};
    launch_events_all<false>(c, s, s.k, pos, tb);
}

namespace {
// each clique of an explicit set adds 1 at prefix length (last position of
// its members) + 1
__global__ void k_clique_events(int64_t c, const int32_t *__restrict__ cl, int k,
                                const int32_t *__restrict__ pos, unsigned long long *hist) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < c;
         q += (int64_t)gridDim.x * blockDim.x) {
        int mx = -1;
        for (int j = 0; j < k; ++j) mx = max(mx, pos[cl[(size_t)q * k + j]]);
        atomicAdd(hist + (mx + 1), 1ull);
    }
}
}  // namespace

// The final step of Alg. 4: nodes sorted by r (non-increasing, ties by id),
// |C_k(V_i) & set| for every prefix from an explicit clique set, and the
// prefix of largest count / i (largest i on ties).  INT64 state.
void extract_from_cliques(const Ctx &c, const StateDev &st, const int32_t *cl, int64_t count,
                          int k, kdss_result *out) {
    const int64_t n = st.n;
    memset(out, 0, sizeof *out);
    out->t_used = st.t;
    out->T = st.t;
    if (n == 0) return;
    const int B = 256;
    DBuf<uint64_t> keys(c, (size_t)n);
    DBuf<int32_t> order(c, (size_t)n);
    unsigned long long mb = 0;
    to_host(c, &mb, st.maxr.p, 1);
    k_keys_u64<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, st.r.p, mb, keys.p, order.p);
    KDSS_LAUNCH_CHECK();
    radix_sort_u64(c, keys.p, order.p, n, {{0, bit_length(mb)}});
    keys.reset();
    DBuf<int32_t> pos(c, (size_t)n);
    k_positions<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, order.p, pos.p);
    KDSS_LAUNCH_CHECK();
    DBuf<unsigned long long> hist(c, (size_t)n + 2);
    zero(c, hist.p, (n + 2) * 8);
    if (count > 0) {
        k_clique_events<<<grid_for(c, count, B, 4), B, 0, c.stream>>>(count, cl, k, pos.p, hist.p);
        KDSS_LAUNCH_CHECK();
    }
    inclusive_scan_u64_async(c, (const uint64_t *)hist.p, (uint64_t *)hist.p, n + 1);
    unsigned long long best = 0;
    long long istar = 0;
    best_prefix(c, n, hist.p, &best, &istar);
    out->istar = istar;
    out->count_lo = best;
    out->density = istar > 0 ? (double)best / (double)istar : 0.0;
    out->upper_bound = st.t > 0 ? (double)mb / st.t : 0.0;
    if (istar > 0) {
        out->ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)istar);
        if (!out->ids) fail(KDSS_ERR_OOM, "host allocation of the result ids");
        to_host(c, out->ids, order.p, (size_t)istar);
        std::sort(out->ids, out->ids + istar);
    }
}

// Extraction in three phases, so that the pairs can come in pieces (the
// streamed solve rebuilds the SCT root range by root range): the order and
// positions from r, the prefix-count increments of each piece of pairs, and
// the scans and the best prefix.
void prefix_begin(const Ctx &c, int64_t n, const StateDev &st, bool wide, PrefixAcc &a) {
    a.n = n;
    a.wide = wide;
    const int B = 256;
    DBuf<uint64_t> keys(c, (size_t)n);
    a.order = DBuf<int32_t>(c, (size_t)n);
    int bits;
    if (st.precision == KDSS_FP32K) {
        DBuf<unsigned long long> mx(c, 1);
        zero(c, mx.p, 8);
        k_max_f32bits<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, st.r32.p, mx.p);
        KDSS_LAUNCH_CHECK();
        unsigned long long mb = 0;
        to_host(c, &mb, mx.p, 1);
        uint32_t m32 = (uint32_t)mb;
        float mf;
        memcpy(&mf, &m32, 4);
        a.rmax = (double)mf;
        k_keys_f32<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, st.r32.p, m32, keys.p, a.order.p);
        bits = bit_length(m32);
    } else {
        unsigned long long mb = 0;
        to_host(c, &mb, st.maxr.p, 1);
        if (st.precision == KDSS_FP64) {
            double md;
            memcpy(&md, &mb, 8);
            a.rmax = st.t > 0 ? md / st.t : 0.0;
            const uint64_t mv = (uint64_t)md;   // an integer below 2^53
            k_keys_f64<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, st.r.p, mv, keys.p, a.order.p);
            bits = bit_length(mv);
        } else {
            a.rmax = st.t > 0 ? (double)mb / st.t : 0.0;
            k_keys_u64<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, st.r.p, mb, keys.p, a.order.p);
            bits = bit_length(mb);
        }
    }
    KDSS_LAUNCH_CHECK();
    radix_sort_u64(c, keys.p, a.order.p, n, {{0, bits}});
    keys.reset();
    a.pos = DBuf<int32_t>(c, (size_t)n);
    k_positions<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, a.order.p, a.pos.p);
    KDSS_LAUNCH_CHECK();
    if (!wide) {
        a.hist = DBuf<unsigned long long>(c, (size_t)n + 2);
        a.fhist = DBuf<unsigned long long>(c, (size_t)n + 2);
        zero(c, a.hist.p, (n + 2) * 8);
        zero(c, a.fhist.p, (n + 2) * 8);
    } else {
        a.hist128 = DBuf<U128>(c, (size_t)n + 2);
        a.fhist128 = DBuf<U128>(c, (size_t)n + 2);
        zero(c, a.hist128.p, (n + 2) * 16);
        zero(c, a.fhist128.p, (n + 2) * 16);
    }
}

void prefix_add(const Ctx &c, const SctDev &s, int k, PrefixAcc &a) {
    if (!a.wide) {
        EventTables<false> tb{s.binom.p, nullptr, a.hist.p, a.fhist.p, nullptr, nullptr};
        launch_events_all<false>(c, s, k, a.pos.p, tb);
    } else {
        EventTables<true> tb{nullptr, s.binom128.p, nullptr, nullptr, a.hist128.p, a.fhist128.p};
        launch_events_all<true>(c, s, k, a.pos.p, tb);
    }
}

void prefix_end(const Ctx &c, PrefixAcc &a, const StateDev &st, kdss_result *out) {
    const int64_t n = a.n;
    long long istar = 0, fi = 0;
    U128 best(0), fbest(0);
    if (!a.wide) {
        inclusive_scan_u64_async(c, (const uint64_t *)a.hist.p, (uint64_t *)a.hist.p, n + 1);
        inclusive_scan_u64_async(c, (const uint64_t *)a.fhist.p, (uint64_t *)a.fhist.p, n + 1);
        unsigned long long b64 = 0, f64 = 0;
        best_prefix(c, n, a.hist.p, &b64, &istar);
        best_prefix(c, n, a.fhist.p, &f64, &fi);
        best = U128(b64, 0ull);
        fbest = U128(f64, 0ull);
    } else {
        inclusive_scan_u128_async(c, a.hist128.p, a.hist128.p, n + 1);
        inclusive_scan_u128_async(c, a.fhist128.p, a.fhist128.p, n + 1);
        best_prefix(c, n, a.hist128.p, &best, &istar);
        best_prefix(c, n, a.fhist128.p, &fbest, &fi);
    }
    out->istar = istar;
    out->count_lo = best.lo;
    out->count_hi = best.hi;
    out->density = istar > 0 ? u128_to_double(best) / (double)istar : 0.0;
    out->upper_bound = a.rmax;
    out->rho_prime = fi > 0 ? u128_to_double(fbest) / (double)fi : 0.0;
    out->gap = a.rmax > 0 ? 1.0 - out->rho_prime / a.rmax : 0.0;
    out->T = st.t;
    out->t_used = st.t;
    if (istar > 0) {
        out->ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)istar);
        if (!out->ids) fail(KDSS_ERR_OOM, "host allocation of the result ids");
        to_host(c, out->ids, a.order.p, (size_t)istar);
        std::sort(out->ids, out->ids + istar);
    }
}

void extract_prefix(const Ctx &c, const SctDev &s, const StateDev &st, kdss_result *out) {
    memset(out, 0, sizeof *out);
    out->t_used = st.t;
    if (s.n == 0) return;
    PrefixAcc a;
    prefix_begin(c, s.n, st, st.ck_hi != 0, a);
    prefix_add(c, s, st.k, a);
    prefix_end(c, a, st, out);
}

}  // namespace kdss
