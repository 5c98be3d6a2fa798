// fw.cu -- steps A4-A5: Frank-Wolfe iterations of PBUpdate over all pairs.
//
// Alg. 2 runs PBUpdate (Alg. 3) for every SCT pair in every iteration.  Here
// all pairs of iteration t read r_{t-1} (synchronous form: the per-pair
// allocations do not depend on the pair order, so integer sums are exact and
// reproducible) and scatter-add their allocation into a delta vector; the
// step kernel then forms r_t = r_{t-1} + delta.  With the cumulative r the FW
// iterate is r / t (step size 1/t, Sec. 3.3).
//
// PBUpdate of one pair (Alg. 3): n_C = C(p, k-h) units; V_h nodes may take up
// to C(p, k-h), V_p nodes up to C(p-1, k-h-1) (C3-C4 of SCT-CP, Lemma 2.6).
// Starting from the lowest plateau of r, the current plateau is raised by
// w = min(smallest remaining cap, gap to the next plateau, floor(n_C/|V_i|));
// capped nodes leave; a plateau that reaches the next one merges with it;
// when floor(n_C/|V_i|) = 0 the remaining units go one each to the lowest-id
// nodes of the plateau (the paper picks them at random; the lowest ids make
// the result deterministic).  Nodes with zero cap never take part.
//
// GPU mapping: a pair is handled by a group of G lanes (G = 8 or 32 by length
// class), each lane holding NPL node slots in registers; node j of the pair
// sits in slot j / G of lane j % G.  Nodes are stored ascending by id, so
// "lowest id" is "lowest slot index" and the remainder ranks come from
// ballots.  Plateau levels, counts and caps are group reductions by
// butterfly shuffles.  Every loop runs warp-uniformly.
//
// The continuous rule (KDSS_FP32K) performs the same walk with real w and no
// remainder on the normalised iterate r/t: iteration t fills n_C / s units
// with caps cap / s on r_{t-1} / (t-1) (s = max(t-1, 1)), which equals the
// cumulative-scale fill divided by s; the allocation is summed with
// error-free (TwoSum) compensated atomics and folded into r/t by a Kahan
// update in the step kernel.
#include <algorithm>
#include <cstdlib>
#include <functional>
#include <type_traits>

#include "fw.cuh"

namespace kdss {

namespace {

constexpr int FW_THREADS = 256;
constexpr unsigned FULL = 0xffffffffu;

template <int G>
__device__ __forceinline__ uint64_t gmin_u64(uint64_t v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        uint64_t t = __shfl_xor_sync(FULL, v, o);
        v = t < v ? t : v;
    }
    return v;
}
template <int G>
__device__ __forceinline__ float gmin_f32(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
template <int G>
__device__ __forceinline__ int gsum_i32(int v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// 1 / s for iteration t = *t_done + 1 of the continuous rule, s = max(t - 1, 1)
// (the step-size schedule is evaluated in FP64).
__device__ __forceinline__ float inv_sigma_of(const int *t_done) {
    const int t = *t_done + 1;
    return (float)(1.0 / (double)(t - 1 > 1 ? t - 1 : 1));
}

template <class RT>
__device__ __forceinline__ uint64_t load_r(const RT *r, int32_t id);
template <>
__device__ __forceinline__ uint64_t load_r<uint64_t>(const uint64_t *r, int32_t id) {
    return __ldg(r + id);
}
template <>
__device__ __forceinline__ uint64_t load_r<double>(const double *r, int32_t id) {
    const uint64_t w = __ldg(reinterpret_cast<const unsigned long long *>(r) + id);
    const int e = (int)(w >> 52) - 1023;  // integer value of the double, integer ops only
    if (e < 0) return 0ull;
    const uint64_t m = (w & ((1ull << 52) - 1)) | (1ull << 52);
    return e >= 52 ? (m << (e - 52)) : (m >> (52 - e));
}
// Asynchronous global -> shared copies (cp.async, 4 or 8 bytes): the data
// does not pass through registers, so a lane can have every copy of a tile in
// flight at once.  Completion is awaited per thread; a __syncwarp() then
// publishes the warp's copies to all its lanes.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Integer value of a double that holds an integer in [0, 2^53), from its bit
// pattern with integer operations only.  Non-negative doubles order like
// their bit patterns, so comparisons may use the raw word; only levels that
// enter arithmetic are converted.
template <class RT>
__device__ __forceinline__ uint64_t level_of(uint64_t w);
template <>
__device__ __forceinline__ uint64_t level_of<uint64_t>(uint64_t w) { return w; }
template <>
__device__ __forceinline__ uint64_t level_of<double>(uint64_t w) {
    const int e = (int)(w >> 52) - 1023;  // 0.0 gives e < 0
    if (e < 0) return 0ull;
    const uint64_t m = (w & ((1ull << 52) - 1)) | (1ull << 52);
    return e >= 52 ? (m << (e - 52)) : (m >> (52 - e));
}

// ---------------------------------------------------------------------------
// Block-local aggregation of the scatter-adds.  Most pairs hand their units
// to a few low-r nodes (on a power-law graph with a planted dense region,
// under 2,000 distinct receivers for 1.6e5 pairs, the busiest node getting
// tens of thousands of adds per iteration), and same-address global atomics
// serialise.  Each block takes a contiguous chunk of pairs (consecutive pairs
// share their root and usually their receiver), adds into a shared-memory
// open-addressing table, and flushes one global atomic per distinct node.
// A crowded table falls back to direct global atomics.
// ---------------------------------------------------------------------------
constexpr int AGG_BITS = 10;
constexpr int AGG_SLOTS = 1 << AGG_BITS;
constexpr int AGG_PROBES = 16;

template <class V>
struct AggTable {
    int32_t key[AGG_SLOTS];
    V val[AGG_SLOTS];
    V comp[sizeof(V) == 4 ? AGG_SLOTS : 1];  // FP32: TwoSum error terms
};

__device__ __forceinline__ unsigned agg_hash(int32_t id) {
    return ((uint32_t)id * 2654435761u) >> (32 - AGG_BITS);
}

template <class V>
__device__ __forceinline__ void agg_init(AggTable<V> &t) {
    for (int i = threadIdx.x; i < AGG_SLOTS; i += blockDim.x) {
        t.key[i] = -1;
        t.val[i] = V(0);
        if (sizeof(V) == 4) t.comp[i] = V(0);
    }
    __syncthreads();
}

__device__ __forceinline__ void gadd(unsigned long long *g, int32_t id, unsigned long long x) {
    atomicAdd(g + id, x);
}
__device__ __forceinline__ void gadd(double *g, int32_t id, double x) { atomicAdd(g + id, x); }
// compensated FP32 add: the exact rounding error of the stored sum goes to gc
__device__ __forceinline__ void gadd_f32(float *g, float *gc, int32_t id, float x) {
    const float old = atomicAdd(g + id, x);
    const float sum = old + x;
    const float bp = sum - old;
    const float e = (old - (sum - bp)) + (x - bp);
    if (e != 0.f) atomicAdd(gc + id, e);
}

// slot of id in the table (inserting it), or -1 when the probe limit is hit
template <class V>
__device__ __forceinline__ int agg_slot(AggTable<V> &t, int32_t id) {
    unsigned sl = agg_hash(id);
    for (int pr = 0; pr < AGG_PROBES; ++pr) {
        const int32_t k = ((volatile int32_t *)t.key)[sl];
        if (k == id) return (int)sl;
        if (k == -1) {
            const int32_t old = atomicCAS(&t.key[sl], -1, id);
            if (old == -1 || old == id) return (int)sl;
        }
        sl = (sl + 1) & (AGG_SLOTS - 1);
    }
    return -1;
}

template <class V>
__device__ __forceinline__ void agg_add(AggTable<V> &t, int32_t id, V x, V *gacc) {
    const int sl = agg_slot(t, id);
    if (sl >= 0) atomicAdd(&t.val[sl], x);
    else gadd(gacc, id, x);
}

__device__ __forceinline__ void agg_add_f32(AggTable<float> &t, int32_t id, float x, float *g,
                                            float *gc) {
    const int sl = agg_slot(t, id);
    if (sl < 0) { gadd_f32(g, gc, id, x); return; }
    const float old = atomicAdd(&t.val[sl], x);
    const float sum = old + x;
    const float bp = sum - old;
    const float e = (old - (sum - bp)) + (x - bp);
    if (e != 0.f) atomicAdd(&t.comp[sl], e);
}

template <class V>
__device__ __forceinline__ void agg_flush(AggTable<V> &t, V *gacc) {
    __syncthreads();
    for (int i = threadIdx.x; i < AGG_SLOTS; i += blockDim.x) {
        const int32_t id = t.key[i];
        if (id >= 0 && t.val[i] != V(0)) gadd(gacc, id, t.val[i]);
    }
}

__device__ __forceinline__ void agg_flush_f32(AggTable<float> &t, float *g, float *gc) {
    __syncthreads();
    for (int i = threadIdx.x; i < AGG_SLOTS; i += blockDim.x) {
        const int32_t id = t.key[i];
        if (id < 0) continue;
        if (t.val[i] != 0.f) gadd_f32(g, gc, id, t.val[i]);
        if (t.comp[i] != 0.f) atomicAdd(gc + id, t.comp[i]);
    }
}

// Accumulator value type of the integer rule for each storage type.
template <class RT> struct AccV;
template <> struct AccV<uint64_t> { using T = unsigned long long; };
template <> struct AccV<double> { using T = double; };

// Rule I PBUpdate of one pair by a group of G lanes (lane gl holds slots
// gl, gl + G, ...): the walk of Alg. 3 with group reductions.  Every lane of
// the warp calls it; `active` is false for lanes whose group has no pair.
// scatter(id, amount) receives each node's allocation.
template <int G, int NPL, class RT, class Scatter>
__device__ __forceinline__ void group_pair_walk(bool active, int64_t q,
                                                const int64_t *__restrict__ pair_off,
                                                const int32_t *__restrict__ nodes,
                                                const uint8_t *__restrict__ hcnt,
                                                const RT *__restrict__ r,
                                                const uint64_t *__restrict__ binom, int bcols,
                                                int k, int *err, Scatter scatter) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned lowmask = (G == 32) ? FULL : ((1u << G) - 1u);
    int64_t off0 = 0;
    int len = 0, h = 0;
    if (active) {
        off0 = pair_off[q];
        len = (int)(pair_off[q + 1] - off0);
        h = hcnt[q];
    }
    // pairs outside P_k (a k-agnostic SCT iterated at k) take no part
    const bool inpk = active && h <= k && k <= len;
    const int p = len - h;
    uint64_t nC = 0, cap_h = 0, cap_p = 0;
    if (inpk) {
        nC = __ldg(binom + (size_t)p * bcols + (k - h));
        cap_h = nC;
        cap_p = (p >= 1 && k - h - 1 >= 0) ? __ldg(binom + (size_t)(p - 1) * bcols + (k - h - 1)) : 0ull;
    }
    uint64_t r0[NPL], cur[NPL], up[NPL];
    int32_t id[NPL];
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
        const int j = s * G + gl;
        const bool valid = inpk && j < len;
        const int32_t raw = valid ? __ldg(nodes + off0 + j) : 0;
        id[s] = raw & 0x7fffffff;
        r0[s] = valid ? load_r<RT>(r, id[s]) : ~0ull;
        up[s] = valid ? (raw < 0 ? cap_h : cap_p) : 0ull;
        cur[s] = r0[s];
    }
    uint64_t rem = inpk ? nC : 0ull;
    uint64_t lev;
    {
        uint64_t m = ~0ull;
#pragma unroll
        for (int s = 0; s < NPL; ++s)
            if (up[s] > 0 && cur[s] < m) m = cur[s];
        lev = gmin_u64<G>(m);
    }
    int guard = 0;
    const int guard_max = 4 * G * NPL + 8;
    while (__any_sync(FULL, rem > 0)) {
        uint64_t nx = ~0ull, mu = ~0ull;
        int na = 0;
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            if (up[s] > 0) {
                if (cur[s] == lev) { ++na; mu = up[s] < mu ? up[s] : mu; }
                else if (cur[s] > lev && cur[s] < nx) nx = cur[s];
            }
        }
        na = gsum_i32<G>(na);
        mu = gmin_u64<G>(mu);
        nx = gmin_u64<G>(nx);
        bool do_rem = false;
        if (rem > 0) {
            if (na == 0) {
                if (nx == ~0ull) { atomicOr(err, DERR_LOGIC); rem = 0; }
                else lev = nx;
            } else {
                const uint64_t gap = nx == ~0ull ? ~0ull : nx - lev;
                uint64_t w = mu < gap ? mu : gap;
                const uint64_t share = rem / (uint64_t)na;
                w = share < w ? share : w;
                if (w > 0) {
#pragma unroll
                    for (int s = 0; s < NPL; ++s)
                        if (up[s] > 0 && cur[s] == lev) { cur[s] += w; up[s] -= w; }
                    rem -= w * (uint64_t)na;
                    lev += w;
                } else {
                    do_rem = true;
                }
            }
        }
        if (__any_sync(FULL, do_rem)) {
            int before = 0;
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                const bool inA = do_rem && up[s] > 0 && cur[s] == lev;
                const unsigned gb = (__ballot_sync(FULL, inA) >> gbase) & lowmask;
                const int rk = before + __popc(gb & ((1u << gl) - 1u));
                if (inA && (uint64_t)rk < rem) { cur[s] += 1; up[s] -= 1; }
                before += __popc(gb);
            }
            if (do_rem) rem = 0;
        }
        if (++guard > guard_max) {
            if (rem > 0) atomicOr(err, DERR_LOGIC);
            break;
        }
    }
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
        const int j = s * G + gl;
        if (inpk && j < len && cur[s] > r0[s])
            scatter(id[s], cur[s] - r0[s]);
    }
}

// Rule I (integer) PBUpdate over the pairs [p_begin, p_end).
template <int G, int NPL, class RT>
__global__ void __launch_bounds__(FW_THREADS)
k_pbupdate_int(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
               const uint8_t *__restrict__ hcnt, int64_t p_begin, int64_t p_end,
               const RT *__restrict__ r, RT *acc, const uint64_t *__restrict__ binom, int bcols,
               int k, const int32_t *list, const int *list_count, int *err) {
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // pairs [p_begin, p_end), or p_begin + list[i] for i < *list_count; each
    // block takes one contiguous chunk
    int64_t np = p_end - p_begin;
    if (list) {
        const int lc = *list_count;
        np = lc < np ? lc : np;
    }
    using AV = typename AccV<RT>::T;
    __shared__ AggTable<AV> tbl;
    agg_init(tbl);
    const int64_t chunk = (np + gridDim.x - 1) / gridDim.x;
    const int64_t cb = blockIdx.x * chunk, ce = cb + chunk < np ? cb + chunk : np;
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    (void)warp; (void)nwarps;
    for (int64_t wb = cb + wib * GPW; wb < ce; wb += wpb * GPW) {
        const int64_t qi = wb + lane / G;
        const bool active = qi < ce;
        const int64_t q = p_begin + (list ? (active ? (int64_t)list[qi] : 0) : qi);
        group_pair_walk<G, NPL, RT>(active, q, pair_off, nodes, hcnt, r, binom, bcols, k, err,
                                    [&](int32_t id, uint64_t x) { agg_add(tbl, id, (AV)x, (AV *)acc); });
    }
    agg_flush(tbl, (AV *)acc);
}

// Warp-segmented aggregation of scatter-adds: lanes holding the same node id
// in consecutive lanes (consecutive pairs usually hand their units to the
// same low-r node) are summed by a segmented scan, and the last lane of each
// run issues one atomic.  Lanes with id < 0 take no part.  Full-warp
// shuffles only; every lane of the warp must call it.
template <class V>
__device__ __forceinline__ void warp_seg_add(int32_t id, V x, V *gacc) {
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int32_t prev = __shfl_up_sync(FULL_, id, 1);
    const bool head = lane == 0 || prev != id;
    const unsigned heads = __ballot_sync(FULL_, head);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const V y = __shfl_up_sync(FULL_, x, o);
        if (lane - o >= start) x += y;
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (tail && id >= 0 && x != V(0)) atomicAdd(gacc + id, x);
}

// The list of pairs the first-step kernels leave to the slow kernels.  The
// unsettled pairs of a tile take their slots with one atomic on the list's
// counter (lane ranks from a ballot), not one atomic each.
// Every lane of the warp calls this; lanes with `want` append `value`.
// Returns the lane's slot (-1 when it appends nothing).
__device__ __forceinline__ int64_t slow_append(bool want, int32_t value, int32_t *slow,
                                               int *slow_count, int64_t cap, int *err) {
    const unsigned FULL_ = 0xffffffffu;
    const unsigned m = __ballot_sync(FULL_, want);
    if (!m) return -1;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if ((threadIdx.x & 31) == leader) base = atomicAdd(slow_count, __popc(m));
    base = __shfl_sync(FULL_, base, leader);
    if (!want) return -1;
    const int64_t slot = (int64_t)base + __popc(m & lanemask_lt());
    if (slot < cap) slow[slot] = value;
    else atomicOr(err, DERR_CAPACITY);
    return slot;
}


// First step of Alg. 3 for pairs of at most 32 nodes.  A warp takes 32
// consecutive pairs: their node ids are copied to shared memory (coalesced)
// and then the r words they address (gathers), both as asynchronous copies so
// that all loads of the tile are in flight at once (the FP32 twin gathers
// through registers, its 4-byte words with the V_h mark in the sign bit);
// then lane i streams pair i from shared memory, finding the lowest level m1
// among the nodes that can receive, the set A of nodes at m1 (slot mask) and
// the next level m2.  With w = floor(n_C/|A|) and R = n_C - w|A|, the walk of
// Alg. 3 ends on this plateau exactly when no node of A reaches its cap and
// the plateau does not reach m2: w < min(cap, m2 - m1) (w <= when R = 0).
// Then every node of A takes w and the R lowest ids one more (one round of
// Alg. 3 plus its remainder step).
// The other pairs (several plateaus or a cap inside the fill) are appended
// to `slow`.
constexpr int FA_WARPS = 4;
constexpr int FA_CAP = 32 * 32;

template <class RT>
__global__ void __launch_bounds__(FA_WARPS * 32)
k_pb_fast(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
          const uint8_t *__restrict__ hcnt, int64_t p_begin, int64_t p_end,
          const RT *__restrict__ r, RT *acc, const uint64_t *__restrict__ binom, int bcols,
          int k, int32_t *slow, int *slow_count, int64_t slow_cap, int *err) {
    __shared__ int32_t sidv[FA_WARPS][FA_CAP];
    __shared__ uint64_t sval[FA_WARPS][FA_CAP];
    using AV = typename AccV<RT>::T;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t np = p_end - p_begin;
    const int64_t ntile = (np + 31) >> 5;
    uint64_t *sv = sval[wib];
    int32_t *sid = sidv[wib];
    for (int64_t tile = blockIdx.x * (int64_t)FA_WARPS + wib; tile < ntile;
         tile += (int64_t)gridDim.x * FA_WARPS) {
        const int64_t qi = tile * 32 + lane;
        const bool valid = qi < np;
        const int64_t q = p_begin + (valid ? qi : np - 1);
        const int64_t myb = pair_off[q], mye = pair_off[q + 1];
        const int64_t B = __shfl_sync(0xffffffffu, myb, 0);
        const int64_t lastq = p_begin + ((tile * 32 + 31 < np) ? tile * 32 + 31 : np - 1);
        const int64_t E = pair_off[lastq + 1];
        const int cnt = (int)(E - B);  // <= 1024 for pairs of <= 32 nodes
        if (cnt > FA_CAP) {             // not a range of short pairs (uniform)
            if (lane == 0) atomicOr(err, DERR_CAPACITY);
            continue;
        }
        // stage: the tile's ids (coalesced), then the r words they address,
        // both as asynchronous copies
        for (int i = lane; i < cnt; i += 32) cp_async4(sid + i, nodes + B + i);
        cp_async_wait_all();
        __syncwarp();
        for (int i = lane; i < cnt; i += 32) cp_async8(sv + i, r + (sid[i] & 0x7fffffff));
        cp_async_wait_all();
        __syncwarp();
        uint32_t rmask = 0;     // receivers (slot bits)
        bool want_slow = false;
        uint64_t w = 0, R = 0;
        int o = 0;
        // pairs outside P_k (a k-agnostic SCT iterated at k) take no part
        const int hq = valid ? (int)hcnt[q] : 0;
        if (valid && hq <= k && k <= (int)(mye - myb)) {
            o = (int)(myb - B);
            const int len = (int)(mye - myb);
            const int h = hq;
            const int p = len - h;
            const uint64_t nC = __ldg(binom + (size_t)p * bcols + (k - h));
            const uint64_t cap_p = (p >= 1 && k - h - 1 >= 0)
                                       ? __ldg(binom + (size_t)(p - 1) * bcols + (k - h - 1)) : 0ull;
            // one branch-free pass over the raw r words (ordered like the
            // levels): lowest level m1 among the nodes that can receive, its
            // node set (mask1, whether it holds a pivot node) and the next
            // level m2.  A pivot node of zero cap (|V_h| = k) reads as ~0 and
            // never receives; hold nodes always can (n_C >= 1).
            const uint64_t pm = cap_p > 0 ? 0ull : ~0ull;
            uint64_t m1 = ~0ull, m2 = ~0ull;
            uint32_t mask1 = 0;
            bool piv1 = false;
            for (int s = 0; s < len; ++s) {
                const uint64_t e = sv[o + s];
                const bool hold = sid[o + s] < 0;
                const uint64_t v = e | (hold ? 0ull : pm);
                const bool lt = v < m1;
                const bool eq = v == m1 && v != ~0ull;
                const uint64_t mn = v < m2 ? v : m2;
                m2 = lt ? m1 : (eq ? m2 : mn);
                m1 = lt ? v : m1;
                const uint32_t bit = 1u << s;
                mask1 = lt ? bit : (eq ? (mask1 | bit) : mask1);
                piv1 = lt ? !hold : (piv1 || (eq && !hold));
            }
            if (mask1) {
                const uint64_t na = (uint64_t)__popc(mask1);
                const uint64_t mu = piv1 ? cap_p : nC;
                const uint64_t gap = m2 == ~0ull ? ~0ull : level_of<RT>(m2) - level_of<RT>(m1);
                w = nC / na;
                R = nC - w * na;
                const uint64_t lim = mu < gap ? mu : gap;
                if (!(R == 0 ? w > lim : w >= lim)) rmask = mask1;  // settled by the first step
                else want_slow = true;
            }
        }
        slow_append(want_slow, (int32_t)qi, slow, slow_count, slow_cap, err);
        // scatter the allocation, one receiver per lane per round
        uint64_t rank = 0;
        while (__any_sync(0xffffffffu, rmask != 0)) {
            int32_t rid = -1;
            AV amount = AV(0);
            if (rmask) {
                const int sl = __ffs(rmask) - 1;
                rmask &= rmask - 1;
                const uint64_t dl = w + (rank < R ? 1ull : 0ull);
                ++rank;
                if (dl) {
                    rid = sid[o + sl] & 0x7fffffff;
                    amount = (AV)dl;
                }
            }
            warp_seg_add<AV>(rid, amount, (AV *)acc);
        }
        __syncwarp();  // sv and sid are rewritten by the next tile
    }
}

// First step on the root-shared form of the SCT (SctDev::rooted()): the
// pairs of a tile come from few roots, and all nodes of a pair lie in its
// root's out-neighbourhood, so the warp gathers the r words of each distinct
// root's neighbourhood once (ids and words staged by asynchronous copies),
// and lane i reads pair i as 16-bit indices into that staged list: the tile
// costs one gather per neighbourhood entry instead of one per pair node, and
// the pair stream is 2 bytes per node instead of 4.  A tile whose
// neighbourhoods do not fit RA_NB entries hands all its pairs to the slow
// kernel, which takes any pair.  The first-step test is k_pb_fast's.
constexpr int RA_WARPS = 4;
constexpr int RA_NB = 768;
constexpr int64_t ROOTED_MIN_BYTES = int64_t(96) << 20;

struct RootedWarpSmem {
    uint64_t nbv[RA_NB];       // r words of the tile's neighbourhoods
    int32_t nbid[RA_NB];       // their original ids
    uint16_t lid[FA_CAP];      // the tile's local indices (V_h mark in bit 15)
};
constexpr size_t RA_SMEM = sizeof(RootedWarpSmem) * RA_WARPS;

template <class RT>
__global__ void __launch_bounds__(RA_WARPS * 32)
k_pb_fast_rooted(const int64_t *__restrict__ pair_off, const uint16_t *__restrict__ lidx,
                 const int32_t *__restrict__ proot, const int64_t *__restrict__ rnb_off,
                 const int32_t *__restrict__ rnb_ids, const uint8_t *__restrict__ hcnt,
                 int64_t p_begin, int64_t p_end, const RT *__restrict__ r, RT *acc,
                 const uint64_t *__restrict__ binom, int bcols, int k, int32_t *slow,
                 int *slow_count, int64_t slow_cap, int *err) {
    extern __shared__ __align__(16) unsigned char ra_smem[];
    using AV = typename AccV<RT>::T;
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    RootedWarpSmem &W = reinterpret_cast<RootedWarpSmem *>(ra_smem)[wib];
    const int64_t np = p_end - p_begin;
    const int64_t ntile = (np + 31) >> 5;
    for (int64_t tile = blockIdx.x * (int64_t)RA_WARPS + wib; tile < ntile;
         tile += (int64_t)gridDim.x * RA_WARPS) {
        const int64_t qi = tile * 32 + lane;
        const bool valid = qi < np;
        const int64_t q = p_begin + (valid ? qi : np - 1);
        const int64_t myb = pair_off[q], mye = pair_off[q + 1];
        const int hq = valid ? (int)hcnt[q] : 0;
        const int32_t root = proot[q];
        const int64_t B = __shfl_sync(FULL_, myb, 0);
        const int64_t E = __shfl_sync(FULL_, mye, 31);
        const int cnt = (int)(E - B);
        if (cnt > FA_CAP) {
            if (lane == 0) atomicOr(err, DERR_CAPACITY);
            continue;
        }
        // distinct roots of the tile: the lowest lane of each root's group
        // leads it; leaders' list sizes, scanned in lane order, place them
        const unsigned grp = __match_any_sync(FULL_, root);
        const int leader = __ffs(grp) - 1;
        const bool lead = lane == leader;
        const int64_t roff = rnb_off[root];
        const int rsz = lead ? (int)(rnb_off[root + 1] - roff) : 0;
        int incl = rsz;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL_, incl, o);
            if (lane >= o) incl += y;
        }
        const int total = __shfl_sync(FULL_, incl, 31);
        const int mybase = __shfl_sync(FULL_, incl - rsz, leader);
        if (total > RA_NB) {   // uniform: the slow kernel takes the whole tile
            const bool inpk = valid && hq <= k && k <= (int)(mye - myb);
            slow_append(inpk, (int32_t)qi, slow, slow_count, slow_cap, err);
            continue;
        }
        // stage the neighbourhoods' ids, and the tile's local indices
        unsigned leaders = __ballot_sync(FULL_, lead);
        while (leaders) {
            const int L = __ffs(leaders) - 1;
            leaders &= leaders - 1;
            const int64_t off = __shfl_sync(FULL_, roff, L);
            const int sz = __shfl_sync(FULL_, rsz, L);
            const int base = __shfl_sync(FULL_, incl - rsz, L);
            for (int i = lane; i < sz; i += 32) cp_async4(W.nbid + base + i, rnb_ids + off + i);
        }
        for (int i = lane; i < cnt; i += 32) W.lid[i] = __ldg(lidx + B + i);
        cp_async_wait_all();
        __syncwarp();
        for (int i = lane; i < total; i += 32) cp_async8(W.nbv + i, r + W.nbid[i]);
        cp_async_wait_all();
        __syncwarp();
        uint32_t rmask = 0;
        bool want_slow = false;
        uint64_t w = 0, R = 0;
        int o = 0;
        if (valid && hq <= k && k <= (int)(mye - myb)) {
            o = (int)(myb - B);
            const int len = (int)(mye - myb);
            const int h = hq;
            const int p = len - h;
            const uint64_t nC = __ldg(binom + (size_t)p * bcols + (k - h));
            const uint64_t cap_p = (p >= 1 && k - h - 1 >= 0)
                                       ? __ldg(binom + (size_t)(p - 1) * bcols + (k - h - 1)) : 0ull;
            const uint64_t pm = cap_p > 0 ? 0ull : ~0ull;
            uint64_t m1 = ~0ull, m2 = ~0ull;
            uint32_t mask1 = 0;
            bool piv1 = false;
            for (int s2 = 0; s2 < len; ++s2) {
                const uint32_t li = W.lid[o + s2];
                const bool hold = (li & 0x8000u) != 0;
                const uint64_t e = W.nbv[mybase + (li & 0x7fffu)];
                const uint64_t v = e | (hold ? 0ull : pm);
                const bool lt = v < m1;
                const bool eq = v == m1 && v != ~0ull;
                const uint64_t mn = v < m2 ? v : m2;
                m2 = lt ? m1 : (eq ? m2 : mn);
                m1 = lt ? v : m1;
                const uint32_t bit = 1u << s2;
                mask1 = lt ? bit : (eq ? (mask1 | bit) : mask1);
                piv1 = lt ? !hold : (piv1 || (eq && !hold));
            }
            if (mask1) {
                const uint64_t na = (uint64_t)__popc(mask1);
                const uint64_t mu = piv1 ? cap_p : nC;
                const uint64_t gap = m2 == ~0ull ? ~0ull : level_of<RT>(m2) - level_of<RT>(m1);
                w = nC / na;
                R = nC - w * na;
                const uint64_t lim = mu < gap ? mu : gap;
                if (!(R == 0 ? w > lim : w >= lim)) rmask = mask1;
                else want_slow = true;
            }
        }
        slow_append(want_slow, (int32_t)qi, slow, slow_count, slow_cap, err);
        uint64_t rank = 0;
        while (__any_sync(FULL_, rmask != 0)) {
            int32_t rid = -1;
            AV amount = AV(0);
            if (rmask) {
                const int sl = __ffs(rmask) - 1;
                rmask &= rmask - 1;
                const uint64_t dl = w + (rank < R ? 1ull : 0ull);
                ++rank;
                if (dl) {
                    rid = W.nbid[mybase + (W.lid[o + sl] & 0x7fffu)];
                    amount = (AV)dl;
                }
            }
            warp_seg_add<AV>(rid, amount, (AV *)acc);
        }
        __syncwarp();
    }
}

// The pairs the first-step kernel left (several plateaus or a cap inside the
// fill), one warp per pair of at most 32 nodes, in closed form.  The
// allocation of Alg. 3 is the integer water level: with
// g(L) = sum_i min(cap_i, max(0, L - r_i)), L* is the largest L with
// g(L) <= n_C, node i gets min(cap_i, max(0, L* - r_i)) and the
// n_C - g(L*) lowest ids among the nodes with r_i <= L* < r_i + cap_i one more.
// g is piecewise linear with breakpoints r_i and r_i + cap_i; lane j
// evaluates g and its right slope s at its own two breakpoints (a pass over
// the pair in shared memory), the largest breakpoint b with g(b) <= n_C wins
// a warp reduction, and L* = b + floor((n_C - g(b)) / s(b)) lies before the
// next breakpoint.  Remainder ranks come from a ballot (lanes are in id order).
constexpr int SB_WARPS = 8;
constexpr int SB_ROUNDS = 24;

// The walk of one pair on levels relative to its lowest receiving node, all
// in 32 bits: lane j holds node j's relative level rl, its cap cl (0: never
// receives) and its id (-1 past the pair); n_C = nC32 < 2^31 and every
// rl < 2^31.  Adds each node's allocation to acc[id].  The walk starts at
// water level L0 with rem0 units left (0 and n_C from the start; a caller
// that already took the first rounds passes the state they reached).
template <class AV>
__device__ __forceinline__ void walk_rel32(uint32_t rl, uint32_t cl, int32_t id, int len,
                                           uint32_t nC32, void *acc, uint64_t *sr_w, int *err,
                                           uint32_t L0 = 0u, uint32_t rem0 = 0xffffffffu) {
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // The walk of Alg. 3 with warp-uniform state: at water level L the
    // receiving nodes are those with rl <= L < rl + cl; the level rises
    // to the next event (a node's level, or a receiving node's level
    // plus cap) while the units last, and stops at
    // L* = L + floor(rem / na) with R = rem mod na units left for the
    // lowest ids receiving at L*.  A level where every node is capped
    // jumps to the next node.  Pairs that cross more than SB_ROUNDS
    // events take the closed form below.
    {
        const uint32_t INF32 = 0xffffffffu;
        // a node that never receives sits at INF32.  Receiving at level L
        // is lo <= L < lo + cl, which is L - lo < cl in wrapping 32-bit
        // arithmetic: rl and cl are below 2^31, so L - lo wraps to at least
        // 2^31 > cl when lo > L (and cl = 0 never holds).
        const uint32_t lo = cl > 0 ? rl : INF32, hi = rl + cl;
        uint32_t L = L0, rem = rem0 == 0xffffffffu ? nC32 : rem0, Ls = 0, R = 0;
        bool done = false;
        for (int round = 0; round < SB_ROUNDS; ++round) {
            const bool act = L - lo < cl;
            const uint32_t na = (uint32_t)__popc(__ballot_sync(FULL_, act));
            const uint32_t ev = __reduce_min_sync(FULL_, act ? hi : (lo > L ? lo : INF32));
            if (na == 0) {
                if (ev == INF32) break;
                L = ev;
                continue;
            }
            // the units end before the next event, or exactly at it
            // (then nothing is left over and L* = ev allocates the
            // same): floor(rem / na) < ev - L, or rem = (ev - L) na,
            // which is rem <= (ev - L) na; one division at the end.
            // With receiving nodes ev is finite (a cap ends below 2^32).
            // One receiving node (the usual case) needs neither the
            // 64-bit product nor the division.
            if (na == 1) {
                if (rem <= ev - L) {
                    Ls = L + rem;
                    R = 0;
                    done = true;
                    break;
                }
                rem -= ev - L;
            } else {
                const uint64_t span = (uint64_t)(ev - L) * na;
                if (rem <= span) {
                    const uint32_t qd = rem / na;
                    Ls = L + qd;
                    R = rem - qd * na;
                    done = true;
                    break;
                }
                rem -= (uint32_t)span;
            }
            L = ev;
        }
        if (done) {
            uint32_t dj = Ls > lo ? min(Ls - lo, cl) : 0u;
            if (R) {   // warp-uniform: the remainder goes to the first R eligible lanes
                const bool elig = Ls - lo < cl;
                const unsigned eb = __ballot_sync(FULL_, elig);
                if (elig && (uint32_t)__popc(eb & lanemask_lt()) < R) dj += 1;
            }
            if (dj) atomicAdd((AV *)acc + id, (AV)dj);
            __syncwarp();
            return;
        }
    }
    // (level, cap) of every node as one 64-bit word; a zero cap adds
    // nothing below (min(d, 0) = 0), so no special case
    uint2 *sp = (uint2 *)sr_w;
    sp[lane] = make_uint2(rl, cl);
    __syncwarp();
    const uint32_t b1 = rl, b2 = rl + cl, lim = nC32 + 1u;
    uint32_t g1 = 0, g2 = 0;
#pragma unroll 4
    for (int i = 0; i < len; ++i) {
        const uint2 e = sp[i];
        if (b1 > e.x) g1 = min(g1 + min(b1 - e.x, e.y), lim);
        if (b2 > e.x) g2 = min(g2 + min(b2 - e.x, e.y), lim);
    }
    uint32_t key = 0, bg = 0;
    int hv = 0;
    if (cl > 0) {
        if (g1 <= nC32) { key = b1; bg = g1; hv = 1; }
        if (g2 <= nC32) { key = b2; bg = g2; hv = 1; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t ok = __shfl_xor_sync(FULL_, key, o);
        const int oh = __shfl_xor_sync(FULL_, hv, o);
        const uint32_t og = __shfl_xor_sync(FULL_, bg, o);
        if (oh && (!hv || ok > key)) { key = ok; hv = 1; bg = og; }
    }
    // right slope of g at the winning breakpoint
    const int bs = __popc(__ballot_sync(FULL_, cl > 0 && key >= rl && key - rl < cl));
    if (!hv || bs <= 0) {
        if (lane == 0) atomicOr(err, DERR_LOGIC);
        return;
    }
    const uint32_t L = key + (nC32 - bg) / (uint32_t)bs;
    uint32_t dj = 0;
    bool elig = false;
    if (cl > 0) {
        if (L > rl) dj = min(L - rl, cl);
        elig = rl <= L && L - rl < cl;
    }
    uint32_t tot = __reduce_add_sync(FULL_, dj);
    const uint32_t R = nC32 - tot;
    const unsigned eb = __ballot_sync(FULL_, elig);
    if (elig && (uint32_t)__popc(eb & lanemask_lt()) < R) dj += 1;
    if (dj) atomicAdd((AV *)acc + id, (AV)dj);
    __syncwarp();
    return;
}

// The water level of one pair of at most 32 nodes by one warp (the closed
// form of Alg. 3's walk): lane j holds node j (raw id with the V_h mark in
// rawc, its integer level rjc); lanes >= len hold nothing.  Used by the slow
// kernel and by the work-queue kernel for the pairs the first step leaves.
// sr_w, sc_w: 32 words of this warp's shared memory each.
template <class AV>
__device__ __forceinline__ void slow_pair_walk(int len, int h, int32_t rawc, uint64_t rjc, int k,
                                               const uint64_t *__restrict__ binom, int bcols,
                                               void *acc, uint64_t *sr_w, uint64_t *sc_w,
                                               int *err) {
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int p = len - h;
    const uint64_t nC = __ldg(binom + (size_t)p * bcols + (k - h));
    const uint64_t cap_p = (p >= 1 && k - h - 1 >= 0)
                               ? __ldg(binom + (size_t)(p - 1) * bcols + (k - h - 1)) : 0ull;
    int32_t id = -1;
    uint64_t rj = 0, cj = 0;
    if (lane < len) {
        id = rawc & 0x7fffffff;
        rj = rjc;
        cj = rawc < 0 ? nC : cap_p;
    }
    // levels relative to the lowest node that can receive: 32-bit when
    // the spread and n_C fit in 31 bits (the usual case).  64-bit min and
    // max as two 32-bit warp reductions (high word, then low word).
    const uint64_t vb = cj > 0 ? rj : ~0ull;
    const uint32_t bh = __reduce_min_sync(FULL_, (uint32_t)(vb >> 32));
    const uint32_t bl = __reduce_min_sync(FULL_, (uint32_t)(vb >> 32) == bh ? (uint32_t)vb : 0xffffffffu);
    const uint64_t base = ((uint64_t)bh << 32) | bl;
    if (__all_sync(FULL_, cj == 0 || rj - base < (1ull << 31)) && nC < (1ull << 31)) {
        const uint32_t rl = cj > 0 ? (uint32_t)(rj - base) : 0u, cl = (uint32_t)cj;
        walk_rel32<AV>(rl, cl, id, len, (uint32_t)nC, acc, sr_w, err);
        return;
    }
    sr_w[lane] = rj;
    sc_w[lane] = cj;
    __syncwarp();
    // g and right slope at my breakpoints rj and rj + cj
    const uint64_t b1 = rj, b2 = rj + cj, lim = nC + 1;
    uint64_t g1 = 0, g2 = 0;
    int s1 = 0, s2 = 0;
    for (int i = 0; i < len; ++i) {
        const uint64_t ri = sr_w[i], ci = sc_w[i];
        if (ci == 0) continue;
        if (b1 > ri) { const uint64_t d = b1 - ri; g1 += d < ci ? d : ci; }
        if (b2 > ri) { const uint64_t d = b2 - ri; g2 += d < ci ? d : ci; }
        g1 = g1 < lim ? g1 : lim;
        g2 = g2 < lim ? g2 : lim;
        s1 += (ri <= b1 && b1 - ri < ci) ? 1 : 0;
        s2 += (ri <= b2 && b2 - ri < ci) ? 1 : 0;
    }
    // best breakpoint of this lane: the larger one with g <= n_C
    uint64_t bb = 0, bg = 0;
    int bs = 0;
    bool have = false;
    if (cj > 0) {
        if (g1 <= nC) { bb = b1; bg = g1; bs = s1; have = true; }
        if (g2 <= nC) { bb = b2; bg = g2; bs = s2; have = true; }
    }
    unsigned long long key = have ? (unsigned long long)bb : 0ull;
    int hv = have ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(FULL_, key, o);
        const int oh = __shfl_xor_sync(FULL_, hv, o);
        const uint64_t og = __shfl_xor_sync(FULL_, bg, o);
        const int os = __shfl_xor_sync(FULL_, bs, o);
        if (oh && (!hv || ok > key)) { key = ok; hv = 1; bg = og; bs = os; }
    }
    if (!hv || bs <= 0) {  // no room below n_C: invariant broken
        if (lane == 0) atomicOr(err, DERR_LOGIC);
        return;
    }
    const uint64_t L = key + (nC - bg) / (uint64_t)bs;
    uint64_t dj = 0;
    bool elig = false;
    if (cj > 0) {
        if (L > rj) { const uint64_t d = L - rj; dj = d < cj ? d : cj; }
        elig = rj <= L && L - rj < cj;
    }
    uint64_t tot = dj;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL_, tot, o);
    const uint64_t R = nC - tot;
    const unsigned eb = __ballot_sync(FULL_, elig);
    if (elig && (uint64_t)__popc(eb & lanemask_lt()) < R) dj += 1;
    if (dj) atomicAdd((AV *)acc + id, (AV)dj);
    __syncwarp();
}

// slow_pair_walk for levels and n_C below 2^31 (the resident kernel's 32-bit
// mode): one 32-bit warp reduction gives the base, no spread test.
template <class AV>
__device__ __forceinline__ void slow_pair_walk32(int len, int h, int32_t rawc, uint32_t lev, int k,
                                                 const uint64_t *__restrict__ binom, int bcols,
                                                 void *acc, uint64_t *sr_w, int *err) {
    const int lane = threadIdx.x & 31;
    const int p = len - h;
    const uint32_t nC = (uint32_t)__ldg(binom + (size_t)p * bcols + (k - h));
    const uint32_t cap_p = (p >= 1 && k - h - 1 >= 0)
                               ? (uint32_t)__ldg(binom + (size_t)(p - 1) * bcols + (k - h - 1)) : 0u;
    int32_t id = -1;
    uint32_t cj = 0;
    if (lane < len) {
        id = rawc & 0x7fffffff;
        cj = rawc < 0 ? nC : cap_p;
    }
    const uint32_t base = __reduce_min_sync(0xffffffffu, cj > 0 ? lev : 0xffffffffu);
    walk_rel32<AV>(cj > 0 ? lev - base : 0u, cj, id, len, nC, acc, sr_w, err);
}

template <class RT, bool PIPE>
__global__ void __launch_bounds__(SB_WARPS * 32, 5)
k_pb_slow(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
          const uint8_t *__restrict__ hcnt, int64_t p_begin, const RT *__restrict__ r,
          RT *acc, const uint64_t *__restrict__ binom, int bcols, int k,
          const int32_t *__restrict__ list, const int *list_count, int64_t list_cap, int *err) {
    __shared__ uint64_t sr[SB_WARPS][32];
    __shared__ uint64_t sc[SB_WARPS][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int64_t np = *list_count;
    np = np < list_cap ? np : list_cap;
    using AVs = typename AccV<RT>::T;
    // PIPE: software pipeline over the warp's pairs li, li + st, li + 2 st,
    // ...  A pair's data is a chain of dependent loads (list entry ->
    // offsets -> node ids -> r words), so each iteration issues the next link
    // for the three following pairs before it works on the current one,
    // whose r words arrived during the previous iteration.  Stage registers:
    // 3 holds the list entry, 2 the offsets, 1 the node id, 0 the r word.
    // Without PIPE each pair loads its own chain (a short list: a few pairs
    // per warp, where the prologue would not pay).
    const int64_t st = (int64_t)gridDim.x * SB_WARPS;
    const int64_t li0 = blockIdx.x * (int64_t)SB_WARPS + wib;
    // a negative entry names no pair and is skipped
    auto pair_of = [&](int64_t x) -> int64_t {
        if (x >= np) return -1;
        const int32_t l = list[x];
        return l >= 0 ? p_begin + l : -1;
    };
    int64_t q3 = -1, q2 = -1, off2 = 0, q1 = -1;
    int len2 = 0, h2 = 0, len1 = 0, h1 = 0, len0 = 0, h0 = 0;
    int32_t raw1 = 0, raw0 = 0;
    uint64_t r0 = 0;
    if constexpr (PIPE) {
        q3 = pair_of(li0 + 3 * st);
        q2 = pair_of(li0 + 2 * st);
        if (q2 >= 0) { off2 = pair_off[q2]; len2 = (int)(pair_off[q2 + 1] - off2); h2 = hcnt[q2]; }
        q1 = pair_of(li0 + st);
        if (q1 >= 0) {
            const int64_t o = pair_off[q1];
            len1 = (int)(pair_off[q1 + 1] - o);
            h1 = hcnt[q1];
            if (lane < len1 && len1 <= 32) raw1 = __ldg(nodes + o + lane);
        }
    }
    for (int64_t li = li0; li < np; li += st) {
        if (!PIPE || li == li0) {  // this pair's own chain
            const int64_t q = pair_of(li);
            len0 = 0;
            if (q >= 0) {
                const int64_t o = pair_off[q];
                len0 = (int)(pair_off[q + 1] - o);
                h0 = hcnt[q];
                if (lane < len0 && len0 <= 32) {
                    raw0 = __ldg(nodes + o + lane);
                    r0 = load_r<RT>(r, raw0 & 0x7fffffff);
                }
            }
        }
        // the current pair
        const int len = len0, h = h0;
        const int32_t rawc = raw0;
        const uint64_t rjc = r0;
        if constexpr (PIPE) {
            // next links of the chain for the following pairs
            const int64_t q4 = pair_of(li + 4 * st);
            int64_t off3 = 0;
            int len3 = 0, h3 = 0;
            if (q3 >= 0) { off3 = pair_off[q3]; len3 = (int)(pair_off[q3 + 1] - off3); h3 = hcnt[q3]; }
            int32_t rawn2 = 0;
            if (q2 >= 0 && lane < len2 && len2 <= 32) rawn2 = __ldg(nodes + off2 + lane);
            uint64_t rn1 = 0;
            if (q1 >= 0 && lane < len1 && len1 <= 32) rn1 = load_r<RT>(r, raw1 & 0x7fffffff);
            // shift the stages
            len0 = len1; h0 = h1; raw0 = raw1; r0 = rn1;
            len1 = len2; h1 = h2; raw1 = rawn2; q1 = q2;
            off2 = off3; len2 = len3; h2 = h3; q2 = q3;
            q3 = q4;
        }
        if (len > 32) {  // uniform: not a short pair
            if (lane == 0) atomicOr(err, DERR_CAPACITY);
            continue;
        }
        if (len == 0) continue;  // an unused slot
        slow_pair_walk<AVs>(len, h, rawc, rjc, k, binom, bcols, acc, sr[wib], sc[wib], err);
    }
}

// ---------------------------------------------------------------------------
// Work-queue iteration (rule I) over one or several SCTs at once.  Persistent
// warps take work items from a device counter: an item is a run of tiles
// (32 consecutive pairs of at most 32 nodes) of one SCT, or a run of its
// longer pairs.  A tile goes through the first step of k_pb_fast, and every
// pair the first step leaves is walked right away by the same warp from the
// tile already staged in shared memory (no slow list, no second read).
// Longer pairs take the group walk, `tpp` lanes per pair.  One launch does
// the PBUpdate pass of every SCT of the batch; the items' size (tiles per
// item) and the lanes per long pair are the tuning knobs.
// ---------------------------------------------------------------------------
constexpr int QW = 4;   // warps per block of the queue kernel

struct QSmem {
    int32_t sid[QW][FA_CAP];
    uint64_t sval[QW][FA_CAP];
    uint64_t sr[QW][32], sc[QW][32];   // walk scratch
};

template <class RT>
__global__ void __launch_bounds__(QW * 32)
k_pb_queue(const QGroup *__restrict__ groups, const QItem *__restrict__ items, int nitems,
           unsigned *cursor, RT *r_all, RT *acc_all, int *err) {
    extern __shared__ __align__(16) unsigned char q_smem[];
    QSmem &S = *reinterpret_cast<QSmem *>(q_smem);
    using AV = typename AccV<RT>::T;
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t *sid = S.sid[wib];
    uint64_t *sv = S.sval[wib];
    while (true) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(cursor, 1u);
        it = __shfl_sync(FULL_, it, 0);
        if (it >= nitems) break;
        const QItem I = items[it];
        const QGroup G = groups[I.g];
        const RT *r = r_all + G.node_off;
        AV *acc = reinterpret_cast<AV *>(acc_all + G.node_off);
        const int k = G.k, bcols = G.bcols;
        const int64_t np = G.short_end;
        for (int64_t tile = I.first; tile < I.first + I.count; ++tile) {
            const int64_t qi = tile * 32 + lane;
            const bool valid = qi < np;
            const int64_t q = valid ? qi : np - 1;
            const int64_t myb = G.pair_off[q], mye = G.pair_off[q + 1];
            const int64_t B = __shfl_sync(FULL_, myb, 0);
            const int64_t E = __shfl_sync(FULL_, mye, 31);
            const int cnt = (int)(E - B);
            if (cnt > FA_CAP) {
                if (lane == 0) atomicOr(err, DERR_CAPACITY);
                continue;
            }
            for (int i = lane; i < cnt; i += 32) cp_async4(sid + i, G.nodes + B + i);
            cp_async_wait_all();
            __syncwarp();
            for (int i = lane; i < cnt; i += 32) cp_async8(sv + i, r + (sid[i] & 0x7fffffff));
            cp_async_wait_all();
            __syncwarp();
            const int o = (int)(myb - B);
            const int len = (int)(mye - myb);
            const int h = valid ? (int)G.h[q] : 0;
            uint32_t rmask = 0;
            bool want_slow = false;
            uint64_t w = 0, R = 0;
            if (valid && h <= k && k <= len) {
                const int p = len - h;
                const uint64_t nC = __ldg(G.binom + (size_t)p * bcols + (k - h));
                const uint64_t cap_p = (p >= 1 && k - h - 1 >= 0)
                                           ? __ldg(G.binom + (size_t)(p - 1) * bcols + (k - h - 1)) : 0ull;
                const uint64_t pm = cap_p > 0 ? 0ull : ~0ull;
                uint64_t m1 = ~0ull, m2 = ~0ull;
                uint32_t mask1 = 0;
                bool piv1 = false;
                for (int s2 = 0; s2 < len; ++s2) {
                    const uint64_t e = sv[o + s2];
                    const bool hold = sid[o + s2] < 0;
                    const uint64_t v = e | (hold ? 0ull : pm);
                    const bool lt = v < m1;
                    const bool eq = v == m1 && v != ~0ull;
                    const uint64_t mn = v < m2 ? v : m2;
                    m2 = lt ? m1 : (eq ? m2 : mn);
                    m1 = lt ? v : m1;
                    const uint32_t bit = 1u << s2;
                    mask1 = lt ? bit : (eq ? (mask1 | bit) : mask1);
                    piv1 = lt ? !hold : (piv1 || (eq && !hold));
                }
                if (mask1) {
                    const uint64_t na = (uint64_t)__popc(mask1);
                    const uint64_t mu = piv1 ? cap_p : nC;
                    const uint64_t gap = m2 == ~0ull ? ~0ull : level_of<RT>(m2) - level_of<RT>(m1);
                    w = nC / na;
                    R = nC - w * na;
                    const uint64_t lim = mu < gap ? mu : gap;
                    if (!(R == 0 ? w > lim : w >= lim)) rmask = mask1;
                    else want_slow = true;
                }
            }
            // the pairs the first step leaves, one by one, by the whole warp
            unsigned um = __ballot_sync(FULL_, want_slow);
            while (um) {
                const int src = __ffs(um) - 1;
                um &= um - 1;
                const int so = __shfl_sync(FULL_, o, src);
                const int sl = __shfl_sync(FULL_, len, src);
                const int shh = __shfl_sync(FULL_, h, src);
                int32_t rawc = 0;
                uint64_t rjc = 0;
                if (lane < sl) {
                    rawc = sid[so + lane];
                    rjc = level_of<RT>(sv[so + lane]);
                }
                slow_pair_walk<AV>(sl, shh, rawc, rjc, k, G.binom, bcols, acc, S.sr[wib], S.sc[wib],
                                   err);
            }
            uint64_t rank = 0;
            while (__any_sync(FULL_, rmask != 0)) {
                int32_t rid = -1;
                AV amount = AV(0);
                if (rmask) {
                    const int sl = __ffs(rmask) - 1;
                    rmask &= rmask - 1;
                    const uint64_t dl = w + (rank < R ? 1ull : 0ull);
                    ++rank;
                    if (dl) {
                        rid = sid[o + sl] & 0x7fffffff;
                        amount = (AV)dl;
                    }
                }
                warp_seg_add<AV>(rid, amount, acc);
            }
            __syncwarp();
        }
    }
}

// The longer pairs of the work-queue pass: items of pairs of one SCT, G lanes
// per pair (NPL slots per lane), GPW = 32 / G pairs per warp at a time.
template <class RT, int G, int NPL>
__global__ void __launch_bounds__(FW_THREADS)
k_pb_queue_long(const QGroup *__restrict__ groups, const QItem *__restrict__ items, int nitems,
                unsigned *cursor, RT *r_all, RT *acc_all, int *err) {
    using AV = typename AccV<RT>::T;
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    while (true) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(cursor, 1u);
        it = __shfl_sync(FULL, it, 0);
        if (it >= nitems) break;
        const QItem I = items[it];
        const QGroup Gd = groups[I.g];
        const RT *r = r_all + Gd.node_off;
        AV *acc = reinterpret_cast<AV *>(acc_all + Gd.node_off);
        for (int64_t q0 = I.first; q0 < I.first + I.count; q0 += GPW) {
            const int64_t q = q0 + lane / G;
            group_pair_walk<G, NPL, RT>(q < I.first + I.count, q, Gd.pair_off, Gd.nodes, Gd.h, r,
                                        Gd.binom, Gd.bcols, Gd.k, err,
                                        [&](int32_t id, uint64_t x) { atomicAdd(acc + id, (AV)x); });
        }
    }
}

// Compensated form of warp_seg_add for FP32: the segmented scan carries a
// TwoSum error term next to each partial sum, and the tail lane adds the sum
// to g[id] with a compensated atomic and the error to gc[id].
__device__ __forceinline__ void warp_seg_add_f32(int32_t id, float x, float *g, float *gc) {
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int32_t prev = __shfl_up_sync(FULL_, id, 1);
    const bool head = lane == 0 || prev != id;
    const unsigned heads = __ballot_sync(FULL_, head);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    float sm = x, cm = 0.f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float ys = __shfl_up_sync(FULL_, sm, o);
        const float yc = __shfl_up_sync(FULL_, cm, o);
        if (lane - o >= start) {
            const float t = sm + ys;
            const float bp = t - sm;
            const float e = (sm - (t - bp)) + (ys - bp);
            sm = t;
            cm = cm + yc + e;
        }
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (tail && id >= 0) {
        if (sm != 0.f) gadd_f32(g, gc, id, sm);
        if (cm != 0.f) atomicAdd(gc + id, cm);
    }
}

// First step of the continuous rule for pairs of at most 32 nodes, staged like
// k_pb_fast: the plateau A at the lowest level m1 takes n_C/s/|A| each when
// that stays within its caps and below the next level m2 (no remainder in the
// continuous rule); otherwise the pair goes to the closed form.  The sign bit
// of a staged value marks V_h nodes (all r/t are >= 0).
template <int DUMMY = 0>
__global__ void __launch_bounds__(FA_WARPS * 32)
k_pb_fast_f32s(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
               const uint8_t *__restrict__ hcnt, int64_t p_begin, int64_t p_end,
               const float *__restrict__ r, float *acc, float *accc,
               const float *__restrict__ binomf, int bcols, int k, const int *t_done,
               int32_t *slow, int *slow_count, int64_t slow_cap, int *err) {
    __shared__ float sval[FA_WARPS][FA_CAP];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t np = p_end - p_begin;
    const int64_t ntile = (np + 31) >> 5;
    const float INF = __int_as_float(0x7f800000);
    const float inv_sigma = inv_sigma_of(t_done);
    float *sv = sval[wib];
    for (int64_t tile = blockIdx.x * (int64_t)FA_WARPS + wib; tile < ntile;
         tile += (int64_t)gridDim.x * FA_WARPS) {
        const int64_t qi = tile * 32 + lane;
        const bool valid = qi < np;
        const int64_t q = p_begin + (valid ? qi : np - 1);
        const int64_t myb = pair_off[q], mye = pair_off[q + 1];
        const int64_t B = __shfl_sync(0xffffffffu, myb, 0);
        const int64_t lastq = p_begin + ((tile * 32 + 31 < np) ? tile * 32 + 31 : np - 1);
        const int cnt = (int)(pair_off[lastq + 1] - B);
        if (cnt > FA_CAP) {
            if (lane == 0) atomicOr(err, DERR_CAPACITY);
            continue;
        }
#pragma unroll 4
        for (int i = lane; i < cnt; i += 32) {
            const int32_t raw = __ldg(nodes + B + i);
            const float v = __ldg(r + (raw & 0x7fffffff));
            sv[i] = raw < 0 ? -v : v;  // -0.0 keeps the mark for v = 0
        }
        __syncwarp();
        uint32_t rmask = 0;
        float share = 0.f;
        int o = 0;
        bool want_slow = false;
        const int hq = valid ? (int)hcnt[q] : 0;   // P_k filter, as k_pb_fast
        if (valid && hq <= k && k <= (int)(mye - myb)) {
            o = (int)(myb - B);
            const int len = (int)(mye - myb);
            const int h = hq;
            const int p = len - h;
            const float nC = __ldg(binomf + (size_t)p * bcols + (k - h)) * inv_sigma;
            const float cap_p = (p >= 1 && k - h - 1 >= 0)
                                    ? __ldg(binomf + (size_t)(p - 1) * bcols + (k - h - 1)) * inv_sigma
                                    : 0.f;
            // branch-free pass as in k_pb_fast; zero-cap pivot nodes read as +inf
            const bool prx = cap_p > 0.f;
            float m1 = INF, m2 = INF;
            uint32_t mask1 = 0;
            bool piv1 = false;
            for (int s2 = 0; s2 < len; ++s2) {
                const float e = sv[o + s2];
                const bool hold = signbit(e);
                const float v = (hold || prx) ? fabsf(e) : INF;
                const bool lt = v < m1;
                const bool eq = v == m1 && v < INF;
                const float mn = fminf(m2, v);
                m2 = lt ? m1 : (eq ? m2 : mn);
                m1 = lt ? v : m1;
                const uint32_t bit = 1u << s2;
                mask1 = lt ? bit : (eq ? (mask1 | bit) : mask1);
                piv1 = lt ? !hold : (piv1 || (eq && !hold));
            }
            if (mask1) {
                const float na = (float)__popc(mask1);
                const float mu = piv1 ? cap_p : nC;
                share = nC / na;
                if (share <= mu && share <= m2 - m1) rmask = mask1;
                else want_slow = true;
            }
        }
        slow_append(want_slow, (int32_t)qi, slow, slow_count, slow_cap, err);
        while (__any_sync(0xffffffffu, rmask != 0)) {
            int32_t rid = -1;
            float amount = 0.f;
            if (rmask) {
                const int sl = __ffs(rmask) - 1;
                rmask &= rmask - 1;
                rid = __ldg(nodes + B + o + sl) & 0x7fffffff;
                amount = share;
            }
            warp_seg_add_f32(rid, amount, acc, accc);
        }
        __syncwarp();
    }
}

// Closed form of the continuous rule for the pairs the first step left, one
// warp per pair of at most 32 nodes, in coordinates relative to the lowest
// active level: L is the water level with g(L) = n_C/s, found from the
// largest breakpoint b with g(b) <= n_C/s as b + (n_C/s - g(b)) / slope(b);
// node j takes min(cap_j, max(0, L - x_j)).
// The continuous water level of one pair of at most 32 nodes by one warp
// (k_pb_slow_f32's walk and closed form): lane j holds node j (raw id with the
// V_h mark in rawc, its r/t value xc); lanes >= len hold nothing.  nC_raw
// and the caps come from the float table, scaled by inv_sigma.  sp_w: 32
// float2 of this warp's shared memory.  add(id, x) receives each node's
// allocation (the compensated global add, or a shared-memory accumulator).
template <class Add>
__device__ __forceinline__ void slow_pair_walk_f32_to(int len, int h, int32_t rawc, float xc, int k,
                                                      const float *__restrict__ binomf, int bcols,
                                                      float inv_sigma, Add add, float2 *sp_w,
                                                      int *err) {
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float INF = __int_as_float(0x7f800000);
    const int p = len - h;
    const float nC = __ldg(binomf + (size_t)p * bcols + (k - h)) * inv_sigma;
    const float cap_p = (p >= 1 && k - h - 1 >= 0)
                            ? __ldg(binomf + (size_t)(p - 1) * bcols + (k - h - 1)) * inv_sigma
                            : 0.f;
    int32_t id = -1;
    float xj = 0.f, cj = 0.f;
    if (lane < len) {
        id = rawc & 0x7fffffff;
        xj = xc;
        cj = rawc < 0 ? nC : cap_p;
    }
    // lowest level among the nodes that can receive (non-negative floats
    // order like their bit patterns: one 32-bit warp reduction)
    const float base = __uint_as_float(
        __reduce_min_sync(FULL_, __float_as_uint(cj > 0.f ? xj : INF)));
    const float xl = cj > 0.f ? xj - base : 0.f;
    // the walk of Alg. 3 in real arithmetic, as in k_pb_slow: the level
    // rises from event to event while the units last and stops at
    // L* = L + rem / na; pairs that cross more than SB_ROUNDS events take
    // the closed form below
    {
        const float top = xl + cj;
        float L = 0.f, rem = nC, Ls = 0.f;
        bool done = false;
        for (int round = 0; round < SB_ROUNDS; ++round) {
            const bool act = cj > 0.f && xl <= L && L < top;
            const int na = __popc(__ballot_sync(FULL_, act));
            const float e1 = (cj > 0.f && xl > L) ? xl : INF;
            const float e2 = act ? top : INF;
            const float ev = __uint_as_float(__reduce_min_sync(FULL_, __float_as_uint(fminf(e1, e2))));
            if (na == 0) {
                if (ev == INF) break;
                L = ev;
                continue;
            }
            const float qd = rem / (float)na;
            if (ev == INF || L + qd <= ev) {
                Ls = L + qd;
                done = true;
                break;
            }
            rem -= (ev - L) * (float)na;
            L = ev;
            if (!(rem > 0.f)) {
                Ls = L;
                done = true;
                break;
            }
        }
        if (done) {
            const float dj = cj > 0.f ? fminf(cj, fmaxf(0.f, Ls - xl)) : 0.f;
            if (dj > 0.f) add(id, dj);
            __syncwarp();
            return;
        }
    }
    sp_w[lane] = make_float2(xl, cj);
    __syncwarp();
    const float b1 = xl, b2 = xl + cj;
    float g1 = 0.f, g2 = 0.f;
#pragma unroll 4
    for (int i = 0; i < len; ++i) {
        const float2 e = sp_w[i];
        g1 += fminf(e.y, fmaxf(0.f, b1 - e.x));
        g2 += fminf(e.y, fmaxf(0.f, b2 - e.x));
    }
    float key = -1.f, bg = 0.f;
    if (cj > 0.f) {
        if (g1 <= nC) { key = b1; bg = g1; }
        if (g2 <= nC) { key = b2; bg = g2; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ok = __shfl_xor_sync(FULL_, key, o);
        const float og = __shfl_xor_sync(FULL_, bg, o);
        if (ok > key) { key = ok; bg = og; }
    }
    if (key < 0.f) {
        if (lane == 0) atomicOr(err, DERR_LOGIC);
        return;
    }
    // right slope at key: nodes with x_j <= key < x_j + c_j, the upper end
    // rounded exactly as the breakpoint b2 was
    const int sl = __popc(__ballot_sync(FULL_, cj > 0.f && key >= xl && key < b2));
    const float L = sl > 0 ? key + (nC - bg) / (float)sl : key;
    const float dj = cj > 0.f ? fminf(cj, fmaxf(0.f, L - xl)) : 0.f;
    if (dj > 0.f) add(id, dj);
    __syncwarp();
}

__device__ __forceinline__ void slow_pair_walk_f32(int len, int h, int32_t rawc, float xc, int k,
                                                   const float *__restrict__ binomf, int bcols,
                                                   float inv_sigma, float *acc, float *accc,
                                                   float2 *sp_w, int *err) {
    slow_pair_walk_f32_to(len, h, rawc, xc, k, binomf, bcols, inv_sigma,
                          [&](int32_t id, float x) { gadd_f32(acc, accc, id, x); }, sp_w, err);
}

template <bool PIPE>
__global__ void __launch_bounds__(SB_WARPS * 32, 5)
k_pb_slow_f32(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
              const uint8_t *__restrict__ hcnt, int64_t p_begin, const float *__restrict__ r,
              float *acc, float *accc, const float *__restrict__ binomf, int bcols, int k,
              const int *t_done, const int32_t *__restrict__ list, const int *list_count,
              int64_t list_cap, int *err) {
    __shared__ float2 sp[SB_WARPS][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const float inv_sigma = inv_sigma_of(t_done);
    int64_t np = *list_count;
    np = np < list_cap ? np : list_cap;
    // the load pipeline of k_pb_slow (PIPE) or one chain per pair
    const int64_t st = (int64_t)gridDim.x * SB_WARPS;
    const int64_t li0 = blockIdx.x * (int64_t)SB_WARPS + wib;
    // a negative entry names no pair and is skipped
    auto pair_of = [&](int64_t x) -> int64_t {
        if (x >= np) return -1;
        const int32_t l = list[x];
        return l >= 0 ? p_begin + l : -1;
    };
    int64_t q3 = -1, q2 = -1, off2 = 0, q1 = -1;
    int len2 = 0, h2 = 0, len1 = 0, h1 = 0, len0 = 0, h0 = 0;
    int32_t raw1 = 0, raw0 = 0;
    float x0 = 0.f;
    if constexpr (PIPE) {
        q3 = pair_of(li0 + 3 * st);
        q2 = pair_of(li0 + 2 * st);
        if (q2 >= 0) { off2 = pair_off[q2]; len2 = (int)(pair_off[q2 + 1] - off2); h2 = hcnt[q2]; }
        q1 = pair_of(li0 + st);
        if (q1 >= 0) {
            const int64_t o = pair_off[q1];
            len1 = (int)(pair_off[q1 + 1] - o);
            h1 = hcnt[q1];
            if (lane < len1 && len1 <= 32) raw1 = __ldg(nodes + o + lane);
        }
    }
    for (int64_t li = li0; li < np; li += st) {
        if (!PIPE || li == li0) {
            const int64_t q = pair_of(li);
            len0 = 0;
            if (q >= 0) {
                const int64_t o = pair_off[q];
                len0 = (int)(pair_off[q + 1] - o);
                h0 = hcnt[q];
                if (lane < len0 && len0 <= 32) {
                    raw0 = __ldg(nodes + o + lane);
                    x0 = __ldg(r + (raw0 & 0x7fffffff));
                }
            }
        }
        const int len = len0, h = h0;
        const int32_t rawc = raw0;
        const float xc = x0;
        if constexpr (PIPE) {
            const int64_t q4 = pair_of(li + 4 * st);
            int64_t off3 = 0;
            int len3 = 0, h3 = 0;
            if (q3 >= 0) { off3 = pair_off[q3]; len3 = (int)(pair_off[q3 + 1] - off3); h3 = hcnt[q3]; }
            int32_t rawn2 = 0;
            if (q2 >= 0 && lane < len2 && len2 <= 32) rawn2 = __ldg(nodes + off2 + lane);
            float xn1 = 0.f;
            if (q1 >= 0 && lane < len1 && len1 <= 32) xn1 = __ldg(r + (raw1 & 0x7fffffff));
            len0 = len1; h0 = h1; raw0 = raw1; x0 = xn1;
            len1 = len2; h1 = h2; raw1 = rawn2; q1 = q2;
            off2 = off3; len2 = len3; h2 = h3; q2 = q3;
            q3 = q4;
        }
        if (len > 32) {
            if (lane == 0) atomicOr(err, DERR_CAPACITY);
            continue;
        }
        if (len == 0) continue;  // an unused slot
        slow_pair_walk_f32(len, h, rawc, xc, k, binomf, bcols, inv_sigma, acc, accc, sp[wib], err);
    }
}

// Rule C PBUpdate of one pair by a group of G lanes (as group_pair_walk):
// the continuous walk relative to the pair's lowest active level; every lane
// of the warp calls it; scatter(id, amount) receives each node's allocation.
template <int G, int NPL, class Scatter>
__device__ __forceinline__ void group_pair_walk_f32(bool active, int64_t q,
                                                    const int64_t *__restrict__ pair_off,
                                                    const int32_t *__restrict__ nodes,
                                                    const uint8_t *__restrict__ hcnt,
                                                    const float *__restrict__ r,
                                                    const float *__restrict__ binomf, int bcols,
                                                    int k, float inv_sigma, int *err,
                                                    Scatter scatter) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const float INF = __int_as_float(0x7f800000);
    int64_t off0 = 0;
    int len = 0, h = 0;
    if (active) {
        off0 = pair_off[q];
        len = (int)(pair_off[q + 1] - off0);
        h = hcnt[q];
    }
    const bool inpk = active && h <= k && k <= len;   // P_k filter, as k_pbupdate_int
    const int p = len - h;
    float nC = 0.f, cap_h = 0.f, cap_p = 0.f;
    if (inpk) {
        nC = __ldg(binomf + (size_t)p * bcols + (k - h)) * inv_sigma;
        cap_h = nC;
        cap_p = (p >= 1 && k - h - 1 >= 0)
                    ? __ldg(binomf + (size_t)(p - 1) * bcols + (k - h - 1)) * inv_sigma
                    : 0.f;
    }
    float r0[NPL], cur[NPL], up[NPL];
    int32_t id[NPL];
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
        const int j = s * G + gl;
        const bool valid = inpk && j < len;
        const int32_t raw = valid ? __ldg(nodes + off0 + j) : 0;
        id[s] = raw & 0x7fffffff;
        r0[s] = valid ? __ldg(r + id[s]) : INF;
        up[s] = valid ? (raw < 0 ? cap_h : cap_p) : 0.f;
        cur[s] = r0[s];
    }
    float rem = inpk ? nC : 0.f;
    // Work relative to the pair's lowest active level, so that the
    // allocation (final level - start) is not a difference of two large
    // values of r.
    float lev = 0.f;
    {
        float m = INF;
#pragma unroll
        for (int s = 0; s < NPL; ++s)
            if (up[s] > 0.f) m = fminf(m, cur[s]);
        const float base = gmin_f32<G>(m);
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            r0[s] = (r0[s] == INF || base == INF) ? INF : r0[s] - base;
            cur[s] = r0[s];
        }
    }
    int guard = 0;
    const int guard_max = 4 * G * NPL + 8;
    while (__any_sync(FULL, rem > 0.f)) {
        float nx = INF, mu = INF;
        int na = 0;
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            if (up[s] > 0.f) {
                if (cur[s] == lev) { ++na; mu = fminf(mu, up[s]); }
                else if (cur[s] > lev) nx = fminf(nx, cur[s]);
            }
        }
        na = gsum_i32<G>(na);
        mu = gmin_f32<G>(mu);
        nx = gmin_f32<G>(nx);
        if (rem > 0.f) {
            if (na == 0) {
                if (nx == INF) { atomicOr(err, DERR_LOGIC); rem = 0.f; }
                else lev = nx;
            } else {
                const float gap = nx - lev;
                const float share = rem / (float)na;
                float w = fminf(mu, gap);
                const bool last = share <= w;
                if (last) w = share;
                const float nl = (!last && w == gap) ? nx : lev + w;
#pragma unroll
                for (int s = 0; s < NPL; ++s)
                    if (up[s] > 0.f && cur[s] == lev) { cur[s] = nl; up[s] -= w; }
                rem = last ? 0.f : rem - w * (float)na;
                if (rem < 0.f) rem = 0.f;
                lev = nl;
            }
        }
        if (++guard > guard_max) break;
    }
#pragma unroll
    for (int s = 0; s < NPL; ++s) {
        const int j = s * G + gl;
        if (inpk && j < len && cur[s] > r0[s])
            scatter(id[s], cur[s] - r0[s]);
    }
}

// Rule C (continuous) PBUpdate on the normalised iterate, FP32.
template <int G, int NPL>
__global__ void __launch_bounds__(FW_THREADS)
k_pbupdate_f32(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
               const uint8_t *__restrict__ hcnt, int64_t p_begin, int64_t p_end,
               const float *__restrict__ r, float *acc, float *accc,
               const float *__restrict__ binomf, int bcols, int k, const int *t_done,
               const int32_t *list, const int *list_count, int *err) {
    constexpr int GPW = 32 / G;
    const float inv_sigma = inv_sigma_of(t_done);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // pairs [p_begin, p_end), or p_begin + list[i] for i < *list_count
    int64_t np = p_end - p_begin;
    if (list) {
        const int lc = *list_count;
        np = lc < np ? lc : np;
    }
    __shared__ AggTable<float> tbl;
    agg_init(tbl);
    const int64_t chunk = (np + gridDim.x - 1) / gridDim.x;
    const int64_t cb = blockIdx.x * chunk, ce = cb + chunk < np ? cb + chunk : np;
    const int wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    (void)warp; (void)nwarps;
    for (int64_t wb = cb + wib * GPW; wb < ce; wb += wpb * GPW) {
        const int64_t qi = wb + lane / G;
        const bool active = qi < ce;
        const int64_t q = p_begin + (list ? (active ? (int64_t)list[qi] : 0) : qi);
        group_pair_walk_f32<G, NPL>(active, q, pair_off, nodes, hcnt, r, binomf, bcols, k, inv_sigma,
                                    err, [&](int32_t id, float x) { agg_add_f32(tbl, id, x, acc, accc); });
    }
    agg_flush_f32(tbl, acc, accc);
}

// The continuous rule (KDSS_FP32K) on the work queue: the first step of
// k_pb_fast_f32s on each tile (r/t words gathered through registers, the V_h
// mark in the sign bit), the pairs it leaves walked by the same warp from the
// staged tile (slow_pair_walk_f32), compensated scatter-adds.
struct QSmemF32 {
    float sval[QW][FA_CAP];
    float2 sp[QW][32];   // walk scratch
};

__global__ void __launch_bounds__(QW * 32)
k_pb_queue_f32(const QGroup *__restrict__ groups, const QItem *__restrict__ items, int nitems,
               unsigned *cursor, const float *__restrict__ r_all, float *acc_all, float *accc_all,
               const int *t_done, int *err) {
    __shared__ QSmemF32 S;
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const float INF = __int_as_float(0x7f800000);
    const float inv_sigma = inv_sigma_of(t_done);
    float *sv = S.sval[wib];
    while (true) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(cursor, 1u);
        it = __shfl_sync(FULL_, it, 0);
        if (it >= nitems) break;
        const QItem I = items[it];
        const QGroup G = groups[I.g];
        const float *r = r_all + G.node_off;
        float *acc = acc_all + G.node_off;
        float *accc = accc_all + G.node_off;
        const int k = G.k, bcols = G.bcols;
        const int64_t np = G.short_end;
        for (int64_t tile = I.first; tile < I.first + I.count; ++tile) {
            const int64_t qi = tile * 32 + lane;
            const bool valid = qi < np;
            const int64_t q = valid ? qi : np - 1;
            const int64_t myb = G.pair_off[q], mye = G.pair_off[q + 1];
            const int64_t B = __shfl_sync(FULL_, myb, 0);
            const int64_t E = __shfl_sync(FULL_, mye, 31);
            const int cnt = (int)(E - B);
            if (cnt > FA_CAP) {
                if (lane == 0) atomicOr(err, DERR_CAPACITY);
                continue;
            }
#pragma unroll 4
            for (int i = lane; i < cnt; i += 32) {
                const int32_t raw = __ldg(G.nodes + B + i);
                const float v = __ldg(r + (raw & 0x7fffffff));
                sv[i] = raw < 0 ? -v : v;  // -0.0 keeps the mark for v = 0
            }
            __syncwarp();
            const int o = (int)(myb - B);
            const int len = (int)(mye - myb);
            const int h = valid ? (int)G.h[q] : 0;
            uint32_t rmask = 0;
            float share = 0.f;
            bool want_slow = false;
            if (valid && h <= k && k <= len) {
                const int p = len - h;
                const float nC = __ldg(G.binomf + (size_t)p * bcols + (k - h)) * inv_sigma;
                const float cap_p = (p >= 1 && k - h - 1 >= 0)
                                        ? __ldg(G.binomf + (size_t)(p - 1) * bcols + (k - h - 1)) * inv_sigma
                                        : 0.f;
                const bool prx = cap_p > 0.f;
                float m1 = INF, m2 = INF;
                uint32_t mask1 = 0;
                bool piv1 = false;
                for (int s2 = 0; s2 < len; ++s2) {
                    const float e = sv[o + s2];
                    const bool hold = signbit(e);
                    const float v = (hold || prx) ? fabsf(e) : INF;
                    const bool lt = v < m1;
                    const bool eq = v == m1 && v < INF;
                    const float mn = fminf(m2, v);
                    m2 = lt ? m1 : (eq ? m2 : mn);
                    m1 = lt ? v : m1;
                    const uint32_t bit = 1u << s2;
                    mask1 = lt ? bit : (eq ? (mask1 | bit) : mask1);
                    piv1 = lt ? !hold : (piv1 || (eq && !hold));
                }
                if (mask1) {
                    const float na = (float)__popc(mask1);
                    const float mu = piv1 ? cap_p : nC;
                    share = nC / na;
                    if (share <= mu && share <= m2 - m1) rmask = mask1;
                    else want_slow = true;
                }
            }
            unsigned um = __ballot_sync(FULL_, want_slow);
            while (um) {
                const int src = __ffs(um) - 1;
                um &= um - 1;
                const int so = __shfl_sync(FULL_, o, src);
                const int sl = __shfl_sync(FULL_, len, src);
                const int shh = __shfl_sync(FULL_, h, src);
                int32_t rawc = 0;
                float xc = 0.f;
                if (lane < sl) {
                    rawc = __ldg(G.nodes + B + so + lane);
                    xc = fabsf(sv[so + lane]);
                }
                slow_pair_walk_f32(sl, shh, rawc, xc, k, G.binomf, bcols, inv_sigma, acc, accc,
                                   S.sp[wib], err);
            }
            while (__any_sync(FULL_, rmask != 0)) {
                int32_t rid = -1;
                float amount = 0.f;
                if (rmask) {
                    const int sl = __ffs(rmask) - 1;
                    rmask &= rmask - 1;
                    rid = __ldg(G.nodes + B + o + sl) & 0x7fffffff;
                    amount = share;
                }
                warp_seg_add_f32(rid, amount, acc, accc);
            }
            __syncwarp();
        }
    }
}

template <int G, int NPL>
__global__ void __launch_bounds__(FW_THREADS)
k_pb_queue_long_f32(const QGroup *__restrict__ groups, const QItem *__restrict__ items, int nitems,
                    unsigned *cursor, const float *__restrict__ r_all, float *acc_all,
                    float *accc_all, const int *t_done, int *err) {
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const float inv_sigma = inv_sigma_of(t_done);
    while (true) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(cursor, 1u);
        it = __shfl_sync(FULL, it, 0);
        if (it >= nitems) break;
        const QItem I = items[it];
        const QGroup Gd = groups[I.g];
        const float *r = r_all + Gd.node_off;
        float *acc = acc_all + Gd.node_off;
        float *accc = accc_all + Gd.node_off;
        for (int64_t q0 = I.first; q0 < I.first + I.count; q0 += GPW) {
            const int64_t q = q0 + lane / G;
            group_pair_walk_f32<G, NPL>(q < I.first + I.count, q, Gd.pair_off, Gd.nodes, Gd.h, r,
                                        Gd.binomf, Gd.bcols, Gd.k, inv_sigma, err,
                                        [&](int32_t id, float x) { gadd_f32(acc, accc, id, x); });
        }
    }
}

// r_t = r_{t-1} + delta (rule I); running max of r for the bound.
template <class RT>
__global__ void k_step_int(int64_t n, RT *r, RT *acc, unsigned long long *maxr, int *slow_count) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *slow_count = 0;  // next iteration's list
    unsigned long long m = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        RT x = r[v] + acc[v];
        r[v] = x;
        acc[v] = RT(0);
        unsigned long long b;
        if constexpr (sizeof(RT) == 8 && RT(0.5) != RT(0)) b = (unsigned long long)__double_as_longlong((double)x);
        else b = (unsigned long long)x;
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(FULL, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(maxr, m);
}

// rhat_t = rhat_{t-1} + (s * a - rhat_{t-1}) / t with Kahan compensation,
// t = *t_done + 1; the last block to finish advances *t_done.
__global__ void k_step_f32(int64_t n, float *r, float *rc, float *a, float *ac, int *t_done,
                           unsigned int *blocks_done, int *slow_count, int advance) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *slow_count = 0;  // next iteration's list
    const int t = *t_done + 1;
    const float sigma = (float)(t - 1 > 1 ? t - 1 : 1);
    const float inv_t = (float)(1.0 / (double)t);
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const float delta = sigma * (a[v] + ac[v]);
        const float rv = r[v];
        const float y = (delta - rv) * inv_t - rc[v];
        const float tt = rv + y;
        rc[v] = (tt - rv) - y;
        r[v] = tt;
        a[v] = 0.f;
        ac[v] = 0.f;
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(blocks_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        *blocks_done = 0u;
        if (advance) *t_done = t;
        __threadfence();
    }
}

// The slow kernels pipeline their loads when the short classes hold at least
// 64 pairs per warp of the grid: about a fifth of the pairs reach the slow
// list, so each warp then walks a dozen or more of them in turn.  With fewer
// the pipeline's prologue costs more than it hides (measured: 5-11% faster
// on 10^7-pair unions, 2-7% slower on the 1.6 x 10^5-pair Chung-Lu graph).
inline bool slow_pipelined(int64_t short_pairs, int grid) {
    return short_pairs >= (int64_t)64 * grid * SB_WARPS;
}

// One iteration's PBUpdate launches.  Pairs of at most 32 nodes (classes
// 0-2, stored contiguously) take the fast first-step kernel, the pairs it
// leaves take the group walk (8 lanes x 4 slots); longer pairs take the
// 32-lane group walk directly.
template <class RT>
void launch_pbupdate_int(const Ctx &c, const SctDev &s, int k, RT *r, RT *acc, int32_t *slow,
                         int *slow_count, int *err, bool force_rooted = false) {
    const int bc = s.bcols();
    const int64_t b = s.class_begin[0], e = s.class_begin[3];
    auto go = [&](auto kern, int G, int64_t pb, int64_t pe, const int32_t *list, const int *lc) {
        const int64_t groups_per_block = (FW_THREADS / 32) * (32 / G);
        int grid = (int)std::min<int64_t>(ceil_div(pe - pb, groups_per_block), (int64_t)c.num_sms * 4);
        kern<<<grid, FW_THREADS, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, pb, pe, r, acc,
                                                s.binom.p, bc, k, list, lc, err);
        KDSS_LAUNCH_CHECK();
    };
    if (e > b) {
        const int64_t tiles = ceil_div(e - b, 32);
        const int64_t cap = slow_list_capacity(e - b, c.num_sms);
        // the root-shared first step where the pair stream exceeds L2 (where
        // each gathered r word costs a DRAM-side sector); the flat one where
        // the SCT stays in L2 and the extra indirection does not pay
        if (s.rooted() && (force_rooted || s.nnodes * (int64_t)sizeof(int32_t) > ROOTED_MIN_BYTES)) {
            static thread_local int attr_dev = -1;
            if (attr_dev != c.device) {
                KDSS_CUDA(cudaFuncSetAttribute(k_pb_fast_rooted<uint64_t>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RA_SMEM));
                KDSS_CUDA(cudaFuncSetAttribute(k_pb_fast_rooted<double>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RA_SMEM));
                attr_dev = c.device;
            }
            int grid = (int)std::min<int64_t>(ceil_div(tiles, RA_WARPS), (int64_t)c.num_sms * 5);
            k_pb_fast_rooted<RT><<<grid, RA_WARPS * 32, RA_SMEM, c.stream>>>(
                s.pair_off.p, s.lidx.p, s.proot.p, s.rnb_off.p, s.rnb_ids.p, s.h.p, b, e, r, acc,
                s.binom.p, bc, k, slow, slow_count, cap, err);
        } else {
            int grid = (int)std::min<int64_t>(ceil_div(tiles, FA_WARPS), (int64_t)c.num_sms * 7);
            k_pb_fast<RT><<<grid, FA_WARPS * 32, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, b, e,
                                                                r, acc, s.binom.p, bc, k, slow,
                                                                slow_count, cap, err);
        }
        KDSS_LAUNCH_CHECK();
        int sgrid = (int)std::min<int64_t>(ceil_div(e - b, SB_WARPS), (int64_t)c.num_sms * 8);
        auto slow_kern = slow_pipelined(e - b, sgrid) ? k_pb_slow<RT, true> : k_pb_slow<RT, false>;
        slow_kern<<<sgrid, SB_WARPS * 32, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, b, r, acc,
                                                         s.binom.p, bc, k, slow, slow_count, cap,
                                                         err);
        KDSS_LAUNCH_CHECK();
    }
    if (s.class_begin[4] > s.class_begin[3])
        go(k_pbupdate_int<32, 8, RT>, 32, s.class_begin[3], s.class_begin[4], nullptr, nullptr);
    if (s.class_begin[5] > s.class_begin[4])
        go(k_pbupdate_int<32, 32, RT>, 32, s.class_begin[4], s.class_begin[5], nullptr, nullptr);
}

void launch_pbupdate_f32_on(const Ctx &c, const SctDev &s, int k, StateDev &st, float *r32,
                            float *a32, float *a32c) {
    const int bc = s.bcols();
    const int64_t b = s.class_begin[0], e = s.class_begin[3];
    auto go = [&](auto kern, int G, int64_t pb, int64_t pe, const int32_t *list, const int *lc) {
        const int64_t groups_per_block = (FW_THREADS / 32) * (32 / G);
        int grid = (int)std::min<int64_t>(ceil_div(pe - pb, groups_per_block), (int64_t)c.num_sms * 4);
        kern<<<grid, FW_THREADS, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, pb, pe, r32,
                                                a32, a32c, s.binomf.p, bc, k,
                                                st.dev_t.p, list, lc, st.err.p);
        KDSS_LAUNCH_CHECK();
    };
    if (e > b) {
        const int64_t tiles = ceil_div(e - b, 32);
        const int64_t cap = slow_list_capacity(e - b, c.num_sms);
        int grid = (int)std::min<int64_t>(ceil_div(tiles, FA_WARPS), (int64_t)c.num_sms * 7);
        k_pb_fast_f32s<<<grid, FA_WARPS * 32, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, b, e,
                                                           r32, a32, a32c, s.binomf.p, bc, k,
                                                           st.dev_t.p, st.ovf_list.p,
                                                           st.ovf_count.p, cap, st.err.p);
        KDSS_LAUNCH_CHECK();
        int sgrid = (int)std::min<int64_t>(ceil_div(e - b, SB_WARPS), (int64_t)c.num_sms * 8);
        auto slow_kern = slow_pipelined(e - b, sgrid) ? k_pb_slow_f32<true> : k_pb_slow_f32<false>;
        slow_kern<<<sgrid, SB_WARPS * 32, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, b, r32,
                                                         a32, a32c, s.binomf.p, bc, k, st.dev_t.p,
                                                         st.ovf_list.p, st.ovf_count.p, cap,
                                                         st.err.p);
        KDSS_LAUNCH_CHECK();
    }
    if (s.class_begin[4] > s.class_begin[3])
        go(k_pbupdate_f32<32, 8>, 32, s.class_begin[3], s.class_begin[4], nullptr, nullptr);
    if (s.class_begin[5] > s.class_begin[4])
        go(k_pbupdate_f32<32, 32>, 32, s.class_begin[4], s.class_begin[5], nullptr, nullptr);
}

void launch_pbupdate_f32(const Ctx &c, const SctDev &s, StateDev &st) {
    launch_pbupdate_f32_on(c, s, st.k, st, st.r32.p, st.a32.p, st.a32c.p);
}

// ---------------------------------------------------------------------------
// Resident iterations (rule I): all T iterations of Alg. 2 in one cooperative
// launch, one block per SM.  The pairs (all of at most 32 nodes) are dealt
// round-robin: pair q goes to block q mod G.  The pairs that need the full
// walk cluster (the roots of a dense region sit next to each other in the
// pair order), and dealing single pairs gives every block an even sample of
// them; contiguous ranges or dealt tiles leave some blocks with far more
// walks than others, and every iteration waits for the slowest block.
//
// A planning kernel gives every block's share its distinct nodes: a hash
// table in shared memory maps each node id to a local index, every pair node
// is rewritten as a 16-bit local index (V_h mark in bit 15), and every pair
// gets its offset in the block's local node list.  The resident kernel copies
// the local indices, offsets and h of its pairs into shared memory once.  An
// iteration then gathers r once per distinct node of the block (the SCT's
// pairs crowd on few nodes: on a 1e5-node power-law graph with a planted
// near-clique the ~16,000 pair nodes of a block name ~200 distinct nodes),
// runs the first step of Alg. 3 over the block's pairs 32 at a time, appends
// the pairs it leaves to a block list, walks that list one pair per warp, and
// adds every allocation into a shared-memory accumulator per distinct node,
// which is flushed with one global atomic per node.
//
// One grid barrier per iteration.  r lives in two copies R[0], R[1] and the
// per-iteration delta in three vectors A[0..2].  Iteration j (0-based) reads
// r_j = R[j%2] + A[(j+2)%3] (the previous delta, not yet folded), adds its
// allocation into A[j%3], and meanwhile every block writes its own node slice
// of R[(j+1)%2] = R[j%2] + A[(j+2)%3] and clears its slice of A[(j+1)%3].
// In iteration j nobody reads R[(j+1)%2] or A[(j+1)%3] (last read in
// iteration j-1) and nobody reads A[j%3] (cleared in iteration j-1, read in
// iteration j+1), so the barrier that ends iteration j is the only ordering
// the buffers need.  After the last iteration each block folds its slice
// into R[0] and clears the deltas, which leaves the state as the per-iteration
// launches do: r_T in R[0], the deltas zero.
// ---------------------------------------------------------------------------
constexpr int RS_WARPS = 32;
constexpr int RS_UCAP = 6144;    // distinct nodes per block share at most
constexpr int RS_HS = 8192;      // hash slots of the planning kernel

struct ResidentArgs {
    const int64_t *pair_off;
    const uint16_t *lidx;    // [nnodes] local index of every pair node in its block
    const uint16_t *loff;    // [npairs] offset of every pair in its block's node list
    const int32_t *uid;      // [G * RS_UCAP] distinct nodes of each block
    const int *plan;         // [2G] distinct nodes, then pair nodes, of each block
    const uint8_t *h;
    int64_t npairs;
    const uint64_t *binom;
    int bcols, k;
    int64_t n;
    uint64_t *R[2];
    uint64_t *A[3];
    unsigned long long *maxr;
    int *err;
    GridBarrier *bar;
    uint64_t timeout_ns;
    int T;
    int ncap, pcap, ucap;    // pair nodes, pairs and distinct nodes of the largest share
};

// Sum of two r words (uint64, or the bits of doubles holding integers).
template <class RT>
__device__ __forceinline__ uint64_t rword_add(uint64_t a, uint64_t b);
template <>
__device__ __forceinline__ uint64_t rword_add<uint64_t>(uint64_t a, uint64_t b) { return a + b; }
template <>
__device__ __forceinline__ uint64_t rword_add<double>(uint64_t a, uint64_t b) {
    return (uint64_t)__double_as_longlong(__longlong_as_double((long long)a) +
                                          __longlong_as_double((long long)b));
}

// walk scratch; the walk list's first-step states (uint4 each); r words,
// accumulators and ids of the distinct nodes; walk-list tags and caps; local
// indices; local pair offsets; the walk list; h
size_t resident_smem_bytes(int ncap, int pcap, int ucap) {
    size_t b = (size_t)RS_WARPS * 64 * sizeof(uint64_t);
    b += (size_t)pcap * sizeof(uint4);
    b += (size_t)ucap * (2 * sizeof(uint64_t) + sizeof(int32_t));
    b += (size_t)pcap * 2 * sizeof(uint32_t);
    b += (size_t)ncap * sizeof(uint16_t);
    b += (size_t)(pcap + 1) * sizeof(uint16_t) + (size_t)pcap * sizeof(uint16_t) + (size_t)pcap;
    return (b + 15) & ~(size_t)15;
}

// Pairs of block b's share: b, b + G, b + 2G, ... below npairs.
__host__ __device__ __forceinline__ int64_t resident_share_pairs(int64_t npairs, int G, int b) {
    return (int64_t)b < npairs ? (npairs - 1 - b) / G + 1 : 0;
}

__device__ __forceinline__ unsigned resident_hash(int32_t id) {
    return ((uint32_t)id * 2654435761u) >> (32 - 13);   // RS_HS = 2^13 slots
}

constexpr size_t RS_PLAN_SMEM = 2 * RS_HS * sizeof(int32_t);

// Planning: for every block's share, the offset of each pair in the share's
// node list (an exclusive scan of the pair lengths, 1024 pairs at a time),
// the distinct nodes, and the local index of every pair node.  plan[b] =
// distinct nodes (RS_UCAP + 1 when the share has more than a block can hold),
// plan[G + b] = pair nodes of the share.
__global__ void __launch_bounds__(1024)
k_resident_plan(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
                int64_t npairs, uint16_t *lidx, uint16_t *loff, int32_t *uid, int *plan) {
    extern __shared__ int32_t rp_smem[];   // RS_HS keys, then RS_HS local indices
    __shared__ int s_nu, s_full, s_run;
    __shared__ int s_wsum[32];
    int32_t *hk = rp_smem, *hv = rp_smem + RS_HS;
    volatile int32_t *vk = hk;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int i = threadIdx.x; i < RS_HS; i += blockDim.x) hk[i] = -1;
    if (threadIdx.x == 0) {
        s_nu = 0;
        s_full = 0;
        s_run = 0;
    }
    __syncthreads();
    const int G = gridDim.x;
    const int64_t np = resident_share_pairs(npairs, G, blockIdx.x);
    int32_t *myuid = uid + (size_t)blockIdx.x * RS_UCAP;
    for (int64_t c0 = 0; c0 < np; c0 += blockDim.x) {   // uniform trip count
        const int64_t j = c0 + threadIdx.x;
        int len = 0;
        int64_t e0 = 0;
        if (j < np) {
            const int64_t q = blockIdx.x + j * G;
            e0 = pair_off[q];
            len = (int)(pair_off[q + 1] - e0);
        }
        // exclusive scan of len over the block
        int x = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[wib] = x;
        __syncthreads();
        if (wib == 0) {
            int t = lane < nwarp ? s_wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            s_wsum[lane] = t;   // inclusive warp totals
        }
        __syncthreads();
        const int excl = s_run + (wib ? s_wsum[wib - 1] : 0) + x - len;
        if (j < np) loff[blockIdx.x + j * G] = (uint16_t)excl;   // shares above 65535 nodes are refused
        __syncthreads();
        if (threadIdx.x == 0) s_run += s_wsum[nwarp - 1];
        // this pair's nodes into the hash table (linear probing, at most every slot)
        for (int y = 0; y < len; ++y) {
            const int32_t id = nodes[e0 + y] & 0x7fffffff;
            unsigned slot = resident_hash(id);
            bool placed = false;
            for (int p = 0; p < RS_HS; ++p) {
                int32_t cur = vk[slot];
                if (cur == -1) {
                    cur = atomicCAS(&hk[slot], -1, id);
                    if (cur == -1) {   // this thread placed id: give it the next index
                        const int li = atomicAdd(&s_nu, 1);
                        if (li < RS_UCAP) {
                            hv[slot] = li;
                            myuid[li] = id;
                        }
                        placed = true;
                        break;
                    }
                }
                if (cur == id) {
                    placed = true;
                    break;
                }
                slot = (slot + 1) & (RS_HS - 1);
            }
            if (!placed) s_full = 1;
        }
        __syncthreads();
    }
    // every pair node as its local index
    for (int64_t j = threadIdx.x; j < np; j += blockDim.x) {
        const int64_t q = blockIdx.x + j * G;
        const int64_t e0 = pair_off[q], e1 = pair_off[q + 1];
        for (int64_t e = e0; e < e1; ++e) {
            const int32_t raw = nodes[e];
            const int32_t id = raw & 0x7fffffff;
            unsigned slot = resident_hash(id);
            int li = RS_UCAP;
            for (int p = 0; p < RS_HS; ++p) {
                const int32_t cur = hk[slot];
                if (cur == id) {
                    li = hv[slot];
                    break;
                }
                if (cur == -1) break;
                slot = (slot + 1) & (RS_HS - 1);
            }
            if (li >= RS_UCAP) s_full = 1;
            lidx[e] = (uint16_t)((li & 0x7fff) | (raw < 0 ? 0x8000 : 0));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        plan[blockIdx.x] = (s_full || s_nu > RS_UCAP) ? RS_UCAP + 1 : s_nu;
        plan[G + blockIdx.x] = s_run;
    }
}

// Lane 0 of a warp waits for walk-list entry wi of iteration tag `tag`:
// returns 1 once it is written, 0 when it will never be (every first-step
// tile is done and the list ended before wi) or when the wait ran past its
// deadline (DERR_TIMEOUT).  The wait sleeps between polls so that the warps
// still in their first-step tiles keep the issue slots.
__device__ __forceinline__ int resident_wait_entry(int wi, int np, unsigned tag, const unsigned *stag,
                                                   const int *s_tdone, const int *s_nslow, int ntile,
                                                   int *err) {
    uint64_t t0 = 0;
    for (unsigned polls = 1;; ++polls) {
        if (wi < np && *(volatile const unsigned *)(stag + wi) == tag) {
            __threadfence_block();
            return 1;
        }
        if (*(volatile const int *)s_tdone == ntile) {
            __threadfence_block();
            if (wi >= *(volatile const int *)s_nslow) return 0;
        }
        if ((polls & 63u) == 0u) {
            const uint64_t t = globaltimer_ns();
            if (t0 == 0) t0 = t;
            else if (t - t0 > 1000000000ull) {   // 1 s: far beyond any iteration
                atomicOr(err, DERR_TIMEOUT);
                return 0;
            }
        }
        __nanosleep(32);
    }
}

// L32: every level stays below 2^31 for the whole launch ((t + T) c_k < 2^31,
// as r_t(u) <= t c_k), so levels, n_C, caps and the per-iteration sums run
// in 32 bits.
template <class RT, bool L32>
__global__ void __launch_bounds__(RS_WARPS * 32, 1) k_fw_resident(const ResidentArgs a) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    __shared__ int s_cursor, s_nslow, s_wcur, s_tdone;
    // the block accumulates in integers (every allocation is an integer
    // below 2^53, and integer adds are native shared-memory atomics) and
    // converts once per node when it flushes; a node's allocations in one
    // iteration sum to at most c_k
    using AV = typename std::conditional<L32, unsigned int, unsigned long long>::type;
    using LT = typename std::conditional<L32, uint32_t, uint64_t>::type;   // levels
    using GV = typename AccV<RT>::T;
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint64_t *wsr = reinterpret_cast<uint64_t *>(rs_smem) + wib * 64;
    uint64_t *wsc = wsr + 32;
    uint4 *sent = reinterpret_cast<uint4 *>(rs_smem + (size_t)RS_WARPS * 64 * sizeof(uint64_t));
    uint64_t *sval = reinterpret_cast<uint64_t *>(sent + a.pcap);
    LT *slev = reinterpret_cast<LT *>(sval);   // integer level of each distinct node
    AV *sacc = reinterpret_cast<AV *>(sval + a.ucap);
    int32_t *suid = reinterpret_cast<int32_t *>(sval + 2 * (size_t)a.ucap);
    unsigned *stag = reinterpret_cast<unsigned *>(suid + a.ucap);
    uint32_t *scap = stag + a.pcap;
    uint16_t *slid = reinterpret_cast<uint16_t *>(scap + a.pcap);
    uint16_t *poff = slid + a.ncap;
    uint16_t *slist = poff + a.pcap + 1;
    uint8_t *hh = reinterpret_cast<uint8_t *>(slist + a.pcap);
    const int G = gridDim.x;
    // this block's distinct nodes, then its pairs b, b + G, ... with their
    // nodes as local indices
    int np = (int)resident_share_pairs(a.npairs, G, blockIdx.x);
    int nu = a.plan[blockIdx.x], nn = a.plan[G + blockIdx.x];
    if (np > a.pcap || nn > a.ncap || nu > a.ucap) {
        // the host sized the shares; a mismatch skips the work but keeps the
        // barriers, so that no other block waits for this one
        if (threadIdx.x == 0) atomicOr(a.err, DERR_CAPACITY);
        nu = 0;
        nn = 0;
        np = 0;
    }
    for (int i = threadIdx.x; i < nu; i += blockDim.x) suid[i] = a.uid[(size_t)blockIdx.x * RS_UCAP + i];
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const int64_t q = blockIdx.x + (int64_t)j * G;
        const int64_t e0 = a.pair_off[q];
        const int len = (int)(a.pair_off[q + 1] - e0);
        const int o = a.loff[q];
        poff[j] = (uint16_t)o;
        hh[j] = a.h[q];
        stag[j] = 0u;   // no entry of this launch yet (tags are iteration + 1)
        if (o + len <= nn)
            for (int x = 0; x < len; ++x) slid[o + x] = a.lidx[e0 + x];
    }
    if (threadIdx.x == 0) poff[np] = (uint16_t)nn;
    __syncthreads();
    const int64_t v0 = a.n * blockIdx.x / G, v1 = a.n * (blockIdx.x + 1) / G;
    const int ntile = (np + 31) >> 5;
    const int k = a.k, bcols = a.bcols;
    for (int j = 0; j < a.T; ++j) {
        const uint64_t *Rc = a.R[j & 1];
        uint64_t *Rn = a.R[(j + 1) & 1];
        const uint64_t *Ap = a.A[(j + 2) % 3];
        uint64_t *Az = a.A[(j + 1) % 3];
        GV *gacc = reinterpret_cast<GV *>(a.A[j % 3]);
        const unsigned tag = (unsigned)j + 1u;
        if (threadIdx.x == 0) {
            s_cursor = 0;
            s_nslow = 0;
            s_wcur = 0;
            s_tdone = 0;
        }
        // r_j of the block's distinct nodes (L2 reads: other blocks wrote them)
        for (int i = threadIdx.x; i < nu; i += blockDim.x) {
            const int32_t u = suid[i];
            slev[i] = (LT)level_of<RT>(rword_add<RT>(__ldcg(Rc + u), __ldcg(Ap + u)));
            sacc[i] = AV(0);
        }
        __syncthreads();
        // One work loop per warp: first-step tiles while any are left, then
        // the walks of the pairs they leave.  A warp out of tiles starts on
        // the walk list while other warps still fill it; every entry carries
        // a tag (the iteration + 1) written after its fields.
        while (true) {
            int ti = 0;
            if (lane == 0) ti = atomicAdd(&s_cursor, 1);
            ti = __shfl_sync(FULL_, ti, 0);
            if (ti >= ntile) break;
            const int qi = ti * 32 + lane;
            const bool valid = qi < np;
            const int o = valid ? poff[qi] : 0;
            const int len = valid ? (int)poff[qi + 1] - o : 0;
            const int h = valid ? (int)hh[qi] : 0;
            uint32_t rmask = 0;
            bool want_slow = false;
            LT w = 0, R = 0, m1 = 0, lim = 0, nC = 0, cap_p = 0, na = 0;
            if (valid && h <= k && k <= len && len <= 32) {
                const int p = len - h;
                nC = (LT)__ldg(a.binom + (size_t)p * bcols + (k - h));
                cap_p = (p >= 1 && k - h - 1 >= 0)
                            ? (LT)__ldg(a.binom + (size_t)(p - 1) * bcols + (k - h - 1)) : LT(0);
                const LT NONE = ~LT(0);
                const LT pm = cap_p > 0 ? LT(0) : NONE;
                LT m2 = NONE;
                m1 = NONE;
                uint32_t mask1 = 0;
                bool piv1 = false;
                for (int s2 = 0; s2 < len; ++s2) {
                    const unsigned l = slid[o + s2];
                    const bool hold = (l & 0x8000u) != 0;
                    const LT v = slev[l & 0x7fffu] | (hold ? LT(0) : pm);
                    const bool lt = v < m1;
                    const bool eq = v == m1 && v != NONE;
                    const LT mn = v < m2 ? v : m2;
                    m2 = lt ? m1 : (eq ? m2 : mn);
                    m1 = lt ? v : m1;
                    const uint32_t bit = 1u << s2;
                    mask1 = lt ? bit : (eq ? (mask1 | bit) : mask1);
                    piv1 = lt ? !hold : (piv1 || (eq && !hold));
                }
                if (mask1) {
                    na = (LT)__popc(mask1);
                    const LT mu = piv1 ? cap_p : nC;
                    const LT gap = m2 == NONE ? NONE : m2 - m1;
                    lim = mu < gap ? mu : gap;
                    // the first round settles the pair iff the units fit
                    // below the next event: n_C <= lim * na
                    bool fits;
                    if constexpr (L32) fits = (uint64_t)nC <= (uint64_t)lim * na;
                    else fits = na == 1 ? nC <= lim : lim >= (nC + na - 1) / na;
                    if (fits) {
                        w = na == 1 ? nC : nC / na;
                        R = nC - w * na;
                        rmask = mask1;
                    } else {
                        want_slow = true;
                    }
                }
            } else if (valid && len > 32) {
                atomicOr(a.err, DERR_CAPACITY);
            }
            const unsigned um = __ballot_sync(FULL_, want_slow);
            if (um) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_nslow, __popc(um));
                base = __shfl_sync(FULL_, base, 0);
                if (want_slow) {
                    const int slot = base + __popc(um & lanemask_lt());
                    slist[slot] = (uint16_t)qi;
                    if constexpr (L32) {
                        // the walk resumes after the first round: level lim
                        // above m1 with n_C - lim * na units left
                        sent[slot] = make_uint4(m1, lim, nC - lim * na, nC);
                        scap[slot] = cap_p;
                    }
                    __threadfence_block();
                    *(volatile unsigned *)(stag + slot) = tag;
                }
            }
            LT rank = 0;
            while (__any_sync(FULL_, rmask != 0)) {
                int32_t rid = -1;
                AV amount = AV(0);
                if (rmask) {
                    const int sl = __ffs(rmask) - 1;
                    rmask &= rmask - 1;
                    const LT dl = w + (rank < R ? LT(1) : LT(0));
                    ++rank;
                    if (dl) {
                        rid = (int32_t)(slid[o + sl] & 0x7fffu);
                        amount = (AV)dl;
                    }
                }
                warp_seg_add<AV>(rid, amount, sacc);
            }
            if (lane == 0) {   // this tile's reservations precede its count
                __threadfence_block();
                atomicAdd(&s_tdone, 1);
            }
        }
        // the walks of the block list, one pair per warp at a time
        while (true) {
            int wi = 0, go = 0;
            if (lane == 0) {
                wi = atomicAdd(&s_wcur, 1);
                go = resident_wait_entry(wi, np, tag, stag, &s_tdone, &s_nslow, ntile, a.err);
            }
            __syncwarp();
            go = __shfl_sync(FULL_, go, 0);
            if (!go) break;
            wi = __shfl_sync(FULL_, wi, 0);
            const int q = slist[wi];
            const int so = poff[q];
            const int sl = (int)poff[q + 1] - so;
            int32_t rawc = 0;
            LT lev = 0;
            if (lane < sl) {
                const unsigned l = slid[so + lane];
                rawc = (int32_t)(l & 0x7fffu) | ((l & 0x8000u) ? (int32_t)0x80000000 : 0);
                lev = slev[l & 0x7fffu];
            }
            if constexpr (L32) {
                const uint4 e = sent[wi];   // m1, level and units after the first round, n_C
                const uint32_t cp = scap[wi];
                int32_t id = -1;
                uint32_t cj = 0;
                if (lane < sl) {
                    id = rawc & 0x7fffffff;
                    cj = rawc < 0 ? e.w : cp;
                }
                walk_rel32<AV>(cj > 0 ? (uint32_t)lev - e.x : 0u, cj, id, sl, e.w, sacc, wsr, a.err,
                               e.y, e.z);
            } else {
                slow_pair_walk<AV>(sl, (int)hh[q], rawc, lev, k, a.binom, bcols, sacc, wsr, wsc, a.err);
            }
        }
        // fold the previous delta into the other copy of r and clear the
        // delta that iteration j + 1 adds into (no other block touches these
        // words in this iteration), while other warps finish their walks
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            __stcg(Rn + v, rword_add<RT>(__ldcg(Rc + v), __ldcg(Ap + v)));
            __stcg(Az + v, 0ull);
        }
        __syncthreads();
        // one global add per distinct node that received units
        for (int i = threadIdx.x; i < nu; i += blockDim.x) {
            const AV x = sacc[i];
            if (x != AV(0)) atomicAdd(gacc + suid[i], (GV)x);
        }
        if (!grid_sync_count(&a.bar->count, (unsigned)(j + 1) * (unsigned)G, a.err, a.timeout_ns)) return;
    }
    // r_T = R[T%2] + A[(T+2)%3] into R[0]; clear the two deltas still set
    const uint64_t *Rc = a.R[a.T & 1];
    uint64_t *Al = a.A[(a.T + 2) % 3], *Ao = a.A[(a.T + 1) % 3];
    unsigned long long m = 0;
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const uint64_t x = rword_add<RT>(__ldcg(Rc + v), __ldcg(Al + v));
        a.R[0][v] = x;
        Al[v] = 0;
        Ao[v] = 0;
        m = x > m ? x : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(FULL_, m, o);
        m = t > m ? t : m;
    }
    if (lane == 0 && m) atomicMax(a.maxr, m);
}

// The continuous rule (FP32, normalised r-hat = r / t with compensated
// sums) in the resident form.  The state is r-hat and its compensation (r,
// rc) and the iteration's allocations and their compensation (a, ac); the
// step after iteration t is the update of k_step_f32.  As in k_fw_resident,
// (r, rc) live in two copies and (a, ac) in three, so that one grid barrier
// per iteration orders everything: iteration j reads r-hat as the step of
// R[j mod 2] with A[(j+2) mod 3] (R[0] itself at j = 0), every block computing
// the same words with the same arithmetic; the owner of a node slice stores
// that step into R[(j+1) mod 2] and clears A[(j+1) mod 3].
struct ResidentArgsF32 {
    const int64_t *pair_off;
    const uint16_t *lidx;
    const uint16_t *loff;
    const int32_t *uid;
    const int *plan;
    const uint8_t *h;
    int64_t npairs;
    const float *binomf;
    int bcols, k;
    int64_t n;
    float *R[2], *RC[2];
    float *A[3], *AC[3];
    int *t_done;
    int *err;
    GridBarrier *bar;
    uint64_t timeout_ns;
    int T;
    int ncap, pcap, ucap;
};

// r-hat and its compensation after step t from (r, rc) and the allocations
// (a, ac) of iteration t: r += (sigma (a + ac) - r) / t, sigma = max(t - 1, 1),
// with the rounding error kept in rc.  Rounded operations only (no fused
// multiply-add), so that every block that computes a node's step gets the
// same words.
__device__ __forceinline__ float2 step_f32(float r, float rc, float a, float ac, int t) {
    const float sigma = (float)(t - 1 > 1 ? t - 1 : 1);
    const float inv_t = (float)(1.0 / (double)t);
    const float delta = __fmul_rn(sigma, __fadd_rn(a, ac));
    const float y = __fsub_rn(__fmul_rn(__fsub_rn(delta, r), inv_t), rc);
    const float tt = __fadd_rn(r, y);
    return make_float2(tt, __fsub_rn(__fsub_rn(tt, r), y));
}

// compensated add into shared accumulators: the exact rounding error of the
// stored sum goes to sc[i]
__device__ __forceinline__ void sadd_f32(float *sa, float *sc, int i, float x) {
    const float old = atomicAdd(sa + i, x);
    const float sum = old + x;
    const float bp = sum - old;
    const float e = (old - (sum - bp)) + (x - bp);
    if (e != 0.f) atomicAdd(sc + i, e);
}

__global__ void __launch_bounds__(RS_WARPS * 32, 1) k_fw_resident_f32(const ResidentArgsF32 a) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    __shared__ int s_cursor, s_nslow, s_wcur, s_tdone;
    const unsigned FULL_ = 0xffffffffu;
    const float INF = __int_as_float(0x7f800000);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    // the layout of k_fw_resident (resident_smem_bytes); the uint4 and cap
    // arrays of the integer walk states are not used here
    float2 *wsp = reinterpret_cast<float2 *>(reinterpret_cast<uint64_t *>(rs_smem) + wib * 64);
    uint4 *sent = reinterpret_cast<uint4 *>(rs_smem + (size_t)RS_WARPS * 64 * sizeof(uint64_t));
    uint64_t *sval = reinterpret_cast<uint64_t *>(sent + a.pcap);
    float *slev = reinterpret_cast<float *>(sval);               // r-hat of each distinct node
    float *sacc = reinterpret_cast<float *>(sval + a.ucap);      // allocations ...
    float *saccc = sacc + a.ucap;                                // ... and their compensation
    int32_t *suid = reinterpret_cast<int32_t *>(sval + 2 * (size_t)a.ucap);
    unsigned *stag = reinterpret_cast<unsigned *>(suid + a.ucap);
    uint32_t *scap = stag + a.pcap;
    uint16_t *slid = reinterpret_cast<uint16_t *>(scap + a.pcap);
    uint16_t *poff = slid + a.ncap;
    uint16_t *slist = poff + a.pcap + 1;
    uint8_t *hh = reinterpret_cast<uint8_t *>(slist + a.pcap);
    const int G = gridDim.x;
    int np = (int)resident_share_pairs(a.npairs, G, blockIdx.x);
    int nu = a.plan[blockIdx.x], nn = a.plan[G + blockIdx.x];
    if (np > a.pcap || nn > a.ncap || nu > a.ucap) {
        if (threadIdx.x == 0) atomicOr(a.err, DERR_CAPACITY);
        nu = 0;
        nn = 0;
        np = 0;
    }
    for (int i = threadIdx.x; i < nu; i += blockDim.x) suid[i] = a.uid[(size_t)blockIdx.x * RS_UCAP + i];
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const int64_t q = blockIdx.x + (int64_t)j * G;
        const int64_t e0 = a.pair_off[q];
        const int len = (int)(a.pair_off[q + 1] - e0);
        const int o = a.loff[q];
        poff[j] = (uint16_t)o;
        hh[j] = a.h[q];
        stag[j] = 0u;
        if (o + len <= nn)
            for (int x = 0; x < len; ++x) slid[o + x] = a.lidx[e0 + x];
    }
    if (threadIdx.x == 0) poff[np] = (uint16_t)nn;
    const int t0 = *(volatile int *)a.t_done;   // iterations done before this launch
    __syncthreads();
    const int64_t v0 = a.n * blockIdx.x / G, v1 = a.n * (blockIdx.x + 1) / G;
    const int ntile = (np + 31) >> 5;
    const int k = a.k, bcols = a.bcols;
    for (int j = 0; j < a.T; ++j) {
        const int t = t0 + j + 1;   // this iteration's number
        const float inv_sigma = (float)(1.0 / (double)(t - 1 > 1 ? t - 1 : 1));
        const float *Rc = a.R[j & 1], *RCc = a.RC[j & 1];
        float *Rn = a.R[(j + 1) & 1], *RCn = a.RC[(j + 1) & 1];
        const float *Ap = a.A[(j + 2) % 3], *ACp = a.AC[(j + 2) % 3];
        float *Az = a.A[(j + 1) % 3], *ACz = a.AC[(j + 1) % 3];
        float *Ag = a.A[j % 3], *ACg = a.AC[j % 3];
        const unsigned tag = (unsigned)j + 1u;
        if (threadIdx.x == 0) {
            s_cursor = 0;
            s_nslow = 0;
            s_wcur = 0;
            s_tdone = 0;
        }
        for (int i = threadIdx.x; i < nu; i += blockDim.x) {
            const int32_t u = suid[i];
            slev[i] = j == 0 ? __ldcg(Rc + u)
                             : step_f32(__ldcg(Rc + u), __ldcg(RCc + u), __ldcg(Ap + u), __ldcg(ACp + u), t - 1).x;
            sacc[i] = 0.f;
            saccc[i] = 0.f;
        }
        __syncthreads();
        // first step of every pair (tiles), then the walks of the pairs it
        // leaves, as in k_fw_resident
        while (true) {
            int ti = 0;
            if (lane == 0) ti = atomicAdd(&s_cursor, 1);
            ti = __shfl_sync(FULL_, ti, 0);
            if (ti >= ntile) break;
            const int qi = ti * 32 + lane;
            const bool valid = qi < np;
            const int o = valid ? poff[qi] : 0;
            const int len = valid ? (int)poff[qi + 1] - o : 0;
            const int h = valid ? (int)hh[qi] : 0;
            uint32_t rmask = 0;
            float share = 0.f;
            bool want_slow = false;
            if (valid && h <= k && k <= len && len <= 32) {
                const int p = len - h;
                const float nC = __ldg(a.binomf + (size_t)p * bcols + (k - h)) * inv_sigma;
                const float cap_p = (p >= 1 && k - h - 1 >= 0)
                                        ? __ldg(a.binomf + (size_t)(p - 1) * bcols + (k - h - 1)) * inv_sigma
                                        : 0.f;
                const bool prx = cap_p > 0.f;   // zero-cap pivot nodes read as +inf
                float m1 = INF, m2 = INF;
                uint32_t mask1 = 0;
                bool piv1 = false;
                for (int s2 = 0; s2 < len; ++s2) {
                    const unsigned l = slid[o + s2];
                    const bool hold = (l & 0x8000u) != 0;
                    const float v = (hold || prx) ? slev[l & 0x7fffu] : INF;
                    const bool lt = v < m1;
                    const bool eq = v == m1 && v < INF;
                    const float mn = fminf(m2, v);
                    m2 = lt ? m1 : (eq ? m2 : mn);
                    m1 = lt ? v : m1;
                    const uint32_t bit = 1u << s2;
                    mask1 = lt ? bit : (eq ? (mask1 | bit) : mask1);
                    piv1 = lt ? !hold : (piv1 || (eq && !hold));
                }
                if (mask1) {
                    const float na = (float)__popc(mask1);
                    const float mu = piv1 ? cap_p : nC;
                    share = nC / na;
                    if (share <= mu && share <= m2 - m1) rmask = mask1;
                    else want_slow = true;
                }
            } else if (valid && len > 32) {
                atomicOr(a.err, DERR_CAPACITY);
            }
            const unsigned um = __ballot_sync(FULL_, want_slow);
            if (um) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_nslow, __popc(um));
                base = __shfl_sync(FULL_, base, 0);
                if (want_slow) {
                    const int slot = base + __popc(um & lanemask_lt());
                    slist[slot] = (uint16_t)qi;
                    __threadfence_block();
                    *(volatile unsigned *)(stag + slot) = tag;
                }
            }
            while (rmask) {
                const int sl = __ffs(rmask) - 1;
                rmask &= rmask - 1;
                sadd_f32(sacc, saccc, (int)(slid[o + sl] & 0x7fffu), share);
            }
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                atomicAdd(&s_tdone, 1);
            }
        }
        while (true) {
            int wi = 0, go = 0;
            if (lane == 0) {
                wi = atomicAdd(&s_wcur, 1);
                go = resident_wait_entry(wi, np, tag, stag, &s_tdone, &s_nslow, ntile, a.err);
            }
            __syncwarp();
            go = __shfl_sync(FULL_, go, 0);
            if (!go) break;
            wi = __shfl_sync(FULL_, wi, 0);
            const int q = slist[wi];
            const int so = poff[q];
            const int sl = (int)poff[q + 1] - so;
            int32_t rawc = 0;
            float xc = 0.f;
            if (lane < sl) {
                const unsigned l = slid[so + lane];
                rawc = (int32_t)(l & 0x7fffu) | ((l & 0x8000u) ? (int32_t)0x80000000 : 0);
                xc = slev[l & 0x7fffu];
            }
            slow_pair_walk_f32_to(sl, (int)hh[q], rawc, xc, k, a.binomf, bcols, inv_sigma,
                                  [&](int32_t li, float x) { sadd_f32(sacc, saccc, li, x); }, wsp, a.err);
        }
        // the owner's slice: the step of iteration t - 1 into the other copy,
        // the allocations of iteration t + 1 cleared
        for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
            float2 nv;
            if (j == 0) nv = make_float2(__ldcg(Rc + v), __ldcg(RCc + v));
            else nv = step_f32(__ldcg(Rc + v), __ldcg(RCc + v), __ldcg(Ap + v), __ldcg(ACp + v), t - 1);
            __stcg(Rn + v, nv.x);
            __stcg(RCn + v, nv.y);
            __stcg(Az + v, 0.f);
            __stcg(ACz + v, 0.f);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nu; i += blockDim.x) {
            const float x = sacc[i], xe = saccc[i];
            const int32_t u = suid[i];
            if (x != 0.f) gadd_f32(Ag, ACg, u, x);
            if (xe != 0.f) atomicAdd(ACg + u, xe);
        }
        if (!grid_sync_count(&a.bar->count, (unsigned)(j + 1) * (unsigned)G, a.err, a.timeout_ns)) return;
    }
    // r-hat after the last step into R[0]; clear the two allocations still set
    const int tl = t0 + a.T;
    const float *Rc = a.R[a.T & 1], *RCc = a.RC[a.T & 1];
    float *Al = a.A[(a.T + 2) % 3], *ACl = a.AC[(a.T + 2) % 3];
    float *Ao = a.A[(a.T + 1) % 3], *ACo = a.AC[(a.T + 1) % 3];
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const float2 nv = step_f32(__ldcg(Rc + v), __ldcg(RCc + v), __ldcg(Al + v), __ldcg(ACl + v), tl);
        a.R[0][v] = nv.x;
        a.RC[0][v] = nv.y;
        Al[v] = 0.f;
        ACl[v] = 0.f;
        Ao[v] = 0.f;
        ACo[v] = 0.f;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.t_done = tl;
}

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};

// Whether the resident launch can run the iterations of this state on s:
// the integer rule, pairs of at most 32 nodes only, and the largest block
// range within one block's shared memory.  Plans once per (state, SCT).
using ResidentKernel = void (*)(ResidentArgs);
ResidentKernel resident_kernel(int precision, bool l32) {
    if (precision == KDSS_FP64) return l32 ? k_fw_resident<double, true> : k_fw_resident<double, false>;
    return l32 ? k_fw_resident<uint64_t, true> : k_fw_resident<uint64_t, false>;
}

bool resident_ready(const Ctx &c, const SctDev &s, StateDev &st) {
    if (st.per_iteration || st.qchunk > 0 || st.force_rooted) return false;
    if (s.npairs <= 0 || s.class_begin[0] != 0 || s.class_begin[3] != s.npairs) return false;
    if (st.res_sct == &s) return st.res_state > 0;
    st.res_sct = &s;
    st.res_state = -1;
    int coop = 0, optin = 0;
    KDSS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c.device));
    KDSS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c.device));
    if (!coop) return false;
    const int G = c.num_sms;
    // cheap rejects: the local indices of the average share, or the largest
    // share's pairs, exceed what a block holds
    if (s.nnodes * (int64_t)sizeof(uint16_t) > (int64_t)G * optin) return false;
    const int64_t pcap = resident_share_pairs(s.npairs, G, 0);
    if (pcap > 65535 || resident_smem_bytes(0, (int)pcap, 0) + 1024 > (size_t)optin) return false;
    // distinct nodes of every share, local indices and offsets
    DBuf<uint16_t> lidx(c, (size_t)std::max<int64_t>(s.nnodes, 1));
    DBuf<uint16_t> loff(c, (size_t)s.npairs);
    DBuf<int32_t> uid(c, (size_t)G * RS_UCAP);
    DBuf<int> plan(c, (size_t)2 * G);
    static thread_local int plan_attr_dev = -1;
    if (plan_attr_dev != c.device) {
        KDSS_CUDA(cudaFuncSetAttribute(k_resident_plan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)RS_PLAN_SMEM));
        plan_attr_dev = c.device;
    }
    k_resident_plan<<<G, 1024, RS_PLAN_SMEM, c.stream>>>(s.pair_off.p, s.nodes.p, s.npairs, lidx.p,
                                                         loff.p, uid.p, plan.p);
    KDSS_LAUNCH_CHECK();
    std::vector<int> hplan((size_t)2 * G);
    to_host(c, hplan.data(), plan.p, (size_t)2 * G);
    int ucap = 0, ncap = 0;
    for (int b = 0; b < G; ++b) {
        ucap = std::max(ucap, hplan[b]);
        ncap = std::max(ncap, hplan[G + b]);
    }
    if (ucap > RS_UCAP || ncap > 65535) return false;
    const size_t smem = resident_smem_bytes(ncap, (int)pcap, ucap);
    if (smem + 1024 > (size_t)optin) return false;   // static shared memory and slack
    int per_sm = 1;
    std::vector<const void *> kerns;
    if (st.precision == KDSS_FP32K) kerns.push_back((const void *)k_fw_resident_f32);
    else kerns = {(const void *)resident_kernel(st.precision, false),
                  (const void *)resident_kernel(st.precision, true)};
    for (const void *kern : kerns) {
        KDSS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int b = 0;
        KDSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, RS_WARPS * 32, smem));
        per_sm = std::min(per_sm, b);
    }
    if (per_sm < 1) return false;
    st.res_lidx = std::move(lidx);
    st.res_loff = std::move(loff);
    st.res_uid = std::move(uid);
    st.res_plan = std::move(plan);
    st.res_ucap = ucap;
    const size_t n = (size_t)std::max<int64_t>(s.n, 1);
    st.res_r1 = DBuf<uint64_t>(c, n);
    st.res_a1 = DBuf<uint64_t>(c, n);
    st.res_a2 = DBuf<uint64_t>(c, n);
    st.res_bar = DBuf<GridBarrier>(c, 1);
    zero(c, st.res_a1.p, n * 8);
    zero(c, st.res_a2.p, n * 8);
    zero(c, st.res_bar.p, sizeof(GridBarrier));
    st.res_ncap = ncap;
    st.res_pcap = (int)pcap;
    st.res_smem = smem;
    st.res_state = 1;
    return true;
}

// T iterations in one resident launch.  With `profile` the launch is timed
// with events; the state's timing then counts it as T iterations (PBUpdate
// and step together).
void fw_run_resident(const Ctx &c, const SctDev &s, StateDev &st, int T, bool profile) {
    ResidentArgs a{};
    a.pair_off = s.pair_off.p;
    a.lidx = st.res_lidx.p;
    a.loff = st.res_loff.p;
    a.uid = st.res_uid.p;
    a.plan = st.res_plan.p;
    a.h = s.h.p;
    a.npairs = s.npairs;
    a.binom = s.binom.p;
    a.bcols = s.bcols();
    a.k = st.k;
    a.n = s.n;
    a.R[0] = st.r.p;
    a.R[1] = st.res_r1.p;
    a.A[0] = st.acc.p;
    a.A[1] = st.res_a1.p;
    a.A[2] = st.res_a2.p;
    a.maxr = st.maxr.p;
    a.err = st.err.p;
    a.bar = st.res_bar.p;
    a.timeout_ns = 20ull * 1000 * 1000 * 1000;   // 20 s per barrier wait
    a.T = T;
    a.ncap = st.res_ncap;
    a.pcap = st.res_pcap;
    a.ucap = st.res_ucap;
    // 32-bit levels when every r_t(u) <= t c_k stays below 2^31
    const long double top = (long double)(st.t + T) *
                            ((long double)st.ck_lo + (long double)st.ck_hi * 18446744073709551616.0L);
    const void *kern = (const void *)resident_kernel(st.precision, top < 2147483648.0L);
    void *args[] = {&a};
    ResidentArgsF32 af{};
    void *args_f[] = {&af};
    if (st.precision == KDSS_FP32K) {
        const size_t n = (size_t)std::max<int64_t>(s.n, 1);   // each extra copy holds 2n floats
        af.pair_off = a.pair_off;
        af.lidx = a.lidx;
        af.loff = a.loff;
        af.uid = a.uid;
        af.plan = a.plan;
        af.h = a.h;
        af.npairs = a.npairs;
        af.binomf = s.binomf.p;
        af.bcols = a.bcols;
        af.k = a.k;
        af.n = a.n;
        af.R[0] = st.r32.p;
        af.RC[0] = st.r32c.p;
        af.R[1] = reinterpret_cast<float *>(st.res_r1.p);
        af.RC[1] = af.R[1] + n;
        af.A[0] = st.a32.p;
        af.AC[0] = st.a32c.p;
        af.A[1] = reinterpret_cast<float *>(st.res_a1.p);
        af.AC[1] = af.A[1] + n;
        af.A[2] = reinterpret_cast<float *>(st.res_a2.p);
        af.AC[2] = af.A[2] + n;
        af.t_done = st.dev_t.p;
        af.err = a.err;
        af.bar = a.bar;
        af.timeout_ns = a.timeout_ns;
        af.T = T;
        af.ncap = a.ncap;
        af.pcap = a.pcap;
        af.ucap = a.ucap;
        kern = (const void *)k_fw_resident_f32;
    }
    // the barrier counter starts from zero in every launch
    zero(c, st.res_bar.p, sizeof(GridBarrier));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (profile) {
        while (st.events.size() < 2) {
            cudaEvent_t e;
            KDSS_CUDA(cudaEventCreate(&e));
            st.events.push_back(e);
        }
        e0 = st.events[0];
        e1 = st.events[1];
        KDSS_CUDA(cudaEventRecord(e0, c.stream));
    }
    KDSS_CUDA(cudaLaunchCooperativeKernel(kern, dim3(c.num_sms), dim3(RS_WARPS * 32),
                                          st.precision == KDSS_FP32K ? args_f : args, st.res_smem,
                                          c.stream));
    KDSS_LAUNCH_CHECK();
    if (profile) KDSS_CUDA(cudaEventRecord(e1, c.stream));
    st.t += T;
    int herr = 0;
    to_host(c, &herr, st.err.p, 1);
    if (profile) {
        float ms = 0.f;
        KDSS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        st.timing.fw_kernel_ms += ms;
        st.timing.fw_launches += T;
    }
    if (herr) {   // the barrier may be left mid-count: plan afresh next time
        zero(c, st.res_bar.p, sizeof(GridBarrier));
        st.res_sct = nullptr;
        if (herr & DERR_TIMEOUT) fail(KDSS_ERR_TIMEOUT, "FW iteration: a grid barrier wait expired");
        fail(KDSS_ERR_CUDA, "FW iteration: water-filling invariant failed on the device");
    }
}

}  // namespace

int64_t slow_list_capacity(int64_t short_pairs, int) { return short_pairs; }

void fw_init(const Ctx &c, const SctDev &s, int precision, StateDev &st, int k) {
    st.precision = precision;
    st.n = s.n;
    st.t = 0;
    st.ctx = c;
    st.k = k < 0 ? s.k : k;
    if (st.k == s.k) {
        st.ck_lo = s.ck_lo;
        st.ck_hi = s.ck_hi;
    } else {
        sct_ck_at(c, s, st.k, st.ck_lo, st.ck_hi);
    }
    const size_t n = (size_t)std::max<int64_t>(s.n, 1);
    if (precision == KDSS_FP32K) {
        st.r32 = DBuf<float>(c, n);
        st.r32c = DBuf<float>(c, n);
        st.a32 = DBuf<float>(c, n);
        st.a32c = DBuf<float>(c, n);
        zero(c, st.r32.p, n * 4);
        zero(c, st.r32c.p, n * 4);
        zero(c, st.a32.p, n * 4);
        zero(c, st.a32c.p, n * 4);
    } else {
        st.r = DBuf<uint64_t>(c, n);
        st.acc = DBuf<uint64_t>(c, n);
        zero(c, st.r.p, n * 8);
        zero(c, st.acc.p, n * 8);
    }
    st.maxr = DBuf<unsigned long long>(c, 1);
    st.err = DBuf<int>(c, 1);
    st.dev_t = DBuf<int>(c, 2);  // [0] iterations done, [1] blocks-done counter
    zero(c, st.dev_t.p, 2 * sizeof(int));
    const int64_t short_pairs = std::max<int64_t>(1, s.class_begin[3] - s.class_begin[0]);
    st.ovf_list = DBuf<int32_t>(c, (size_t)slow_list_capacity(short_pairs, c.num_sms));
    st.ovf_count = DBuf<int>(c, 1);
    zero(c, st.ovf_count.p, sizeof(int));
    zero(c, st.maxr.p, 8);
    zero(c, st.err.p, 4);
}

namespace {

void enqueue_pbupdate(const Ctx &c, const SctDev &s, StateDev &st) {
    if (st.qchunk > 0) {
        queue_enqueue(c, st.qplan, st);
    } else if (st.precision == KDSS_FP32K) {
        launch_pbupdate_f32(c, s, st);
    } else if (st.precision == KDSS_FP64) {
        launch_pbupdate_int<double>(c, s, st.k, (double *)st.r.p, (double *)st.acc.p, st.ovf_list.p,
                                    st.ovf_count.p, st.err.p, st.force_rooted);
    } else {
        launch_pbupdate_int<uint64_t>(c, s, st.k, st.r.p, st.acc.p, st.ovf_list.p, st.ovf_count.p,
                                      st.err.p, st.force_rooted);
    }
}

void enqueue_step(const Ctx &c, const SctDev &s, StateDev &st) {
    const int64_t n = s.n;
    if (n <= 0) return;
    const int B = 256;
    const int sgrid = grid_for(c, n, B, 4);
    if (st.precision == KDSS_FP32K) {
        k_step_f32<<<sgrid, B, 0, c.stream>>>(n, st.r32.p, st.r32c.p, st.a32.p, st.a32c.p,
                                             st.dev_t.p, (unsigned int *)(st.dev_t.p + 1),
                                             st.ovf_count.p, 1);
    } else if (st.precision == KDSS_FP64) {
        k_step_int<double><<<sgrid, B, 0, c.stream>>>(n, (double *)st.r.p, (double *)st.acc.p,
                                                      st.maxr.p, st.ovf_count.p);
    } else {
        k_step_int<uint64_t><<<sgrid, B, 0, c.stream>>>(n, st.r.p, st.acc.p, st.maxr.p,
                                                        st.ovf_count.p);
    }
    KDSS_LAUNCH_CHECK();
}

// Capture `fn` on a private stream into an executable graph; returns the
// number of kernels it holds.
template <class F>
long long capture(const Ctx &c, cudaGraphExec_t *exec, F fn) {
    cudaStream_t cap = nullptr;
    KDSS_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    Ctx cc = c;
    cc.stream = cap;
    const long long before = thread_launches();
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        try {
            fn(cc);
        } catch (...) {
            cudaStreamEndCapture(cap, &g);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
            throw;
        }
        e = cudaStreamEndCapture(cap, &g);
    }
    const long long nk = thread_launches() - before;
    add_launches(-nk);  // captured, not run
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    check_cuda(e, "FW graph capture", __FILE__, __LINE__);
    return nk;
}

}  // namespace

StateDev::~StateDev() {
    release_graphs();
    for (cudaEvent_t e : events) cudaEventDestroy(e);
}

void StateDev::release_graphs() {
    for (cudaGraphExec_t *g : {&g_iter, &g_pb, &g_step})
        if (*g) { cudaGraphExecDestroy(*g); *g = nullptr; }
    graph_sct = nullptr;
}

constexpr int FW_PROFILE_EVERY = 8;

void fw_run(const Ctx &c, const SctDev &s, StateDev &st, int T, bool profile) {
    if (T <= 0) return;
    // exactness of the cumulative r: r_t(u) <= t * c_k
    if (st.precision != KDSS_FP32K) {
        const long double lim = st.precision == KDSS_INT64 ? 9.2e18L : 9.007199254740992e15L;
        const long double ck = (long double)st.ck_lo + (long double)st.ck_hi * 18446744073709551616.0L;
        if ((long double)(st.t + T) * ck >= lim)
            fail(KDSS_ERR_OVERFLOW, "T * c_k leaves the exact range of r");
    }
    if (resident_ready(c, s, st)) {
        fw_run_resident(c, s, st, T, profile);
        return;
    }
    // One iteration as CUDA graphs (PBUpdate, step, and both), captured once
    // per (state, SCT) and replayed T times on the caller's stream.
    if (st.graph_sct != &s) {
        st.release_graphs();
        if (st.qchunk > 0) queue_plan(c, {{&s, 0}}, st.qchunk, st.qtpp, st.qplan, st.k);
        st.nk_pb = capture(c, &st.g_pb, [&](const Ctx &cc) { enqueue_pbupdate(cc, s, st); });
        st.nk_step = capture(c, &st.g_step, [&](const Ctx &cc) { enqueue_step(cc, s, st); });
        capture(c, &st.g_iter, [&](const Ctx &cc) {
            enqueue_pbupdate(cc, s, st);
            enqueue_step(cc, s, st);
        });
        st.graph_sct = &s;
    }
    // event pool kept in the state (creating events per call costs host time)
    if (profile) {
        while (st.events.size() < (size_t)T * 4) {
            cudaEvent_t e;
            KDSS_CUDA(cudaEventCreate(&e));
            st.events.push_back(e);
        }
    }
    // Profiling times every FW_PROFILE_EVERY-th iteration (its PBUpdate pass
    // and its step as separate graphs between events); the others run the
    // fused graph, so that timing does not slow the run it measures.
    std::vector<cudaEvent_t> &ev = st.events;
    for (int it = 0; it < T; ++it) {
        if (profile && (st.t + it) % FW_PROFILE_EVERY == 0) {
            KDSS_CUDA(cudaEventRecord(ev[4 * it], c.stream));
            KDSS_CUDA(cudaGraphLaunch(st.g_pb, c.stream));
            KDSS_CUDA(cudaEventRecord(ev[4 * it + 1], c.stream));
            KDSS_CUDA(cudaEventRecord(ev[4 * it + 2], c.stream));
            KDSS_CUDA(cudaGraphLaunch(st.g_step, c.stream));
            KDSS_CUDA(cudaEventRecord(ev[4 * it + 3], c.stream));
        } else {
            KDSS_CUDA(cudaGraphLaunch(st.g_iter, c.stream));
        }
        add_launches(st.nk_pb + st.nk_step);
    }
    st.t += T;
    int herr = 0;
    to_host(c, &herr, st.err.p, 1);
    if (profile) {
        for (int it = 0; it < T; ++it) {
            if ((st.t - T + it) % FW_PROFILE_EVERY != 0) continue;
            float a = 0.f, b2 = 0.f;
            KDSS_CUDA(cudaEventElapsedTime(&a, ev[4 * it], ev[4 * it + 1]));
            KDSS_CUDA(cudaEventElapsedTime(&b2, ev[4 * it + 2], ev[4 * it + 3]));
            st.timing.fw_kernel_ms += a;
            st.timing.step_kernel_ms += b2;
            st.timing.fw_launches += 1;
            st.timing.step_launches += 1;
        }
    }
    if (herr) fail(KDSS_ERR_CUDA, "FW iteration: water-filling invariant failed on the device");
}

// T rule-I iterations on caller-given device memory: r (uint64, cumulative)
// and the scratch the iterations need -- the per-iteration delta `acc` (n
// entries, zero on entry), the list of pairs left to the closed form `slow`
// (one entry per pair of at most 32 nodes), its counter, the error word and
// the running max of r.  Plain launches on c.stream: no allocation, no graph.
void fw_run_external(const Ctx &c, const SctDev &s, uint64_t *r, uint64_t *acc, int32_t *slow,
                     int *slow_count, int *err, unsigned long long *maxr, int T) {
    const int64_t n = s.n;
    const int B = 256;
    const int sgrid = grid_for(c, n, B, 4);
    for (int it = 0; it < T; ++it) {
        launch_pbupdate_int<uint64_t>(c, s, s.k, r, acc, slow, slow_count, err);
        if (n > 0) {
            k_step_int<uint64_t><<<sgrid, B, 0, c.stream>>>(n, r, acc, maxr, slow_count);
            KDSS_LAUNCH_CHECK();
        }
    }
}

// ---- in-place iterations (KDSS_FLAG_ASYNC) ----
//
// The PBUpdate launches of one iteration with the delta vector replaced by r
// itself: every pair's allocation lands in r at once and pairs that read r
// later see it (Alg. 2's in-place update, in the order the GPU happens to
// run the pairs).  Iterations are replayed from one CUDA graph holding the
// slow-list reset and the PBUpdate launches; the running max of r for the
// bound is taken once at the end (r only grows), by the step kernel over a
// zero delta.
void fw_run_async(const Ctx &c, const SctDev &s, StateDev &st, int T) {
    if (T <= 0) return;
    if (st.precision == KDSS_FP32K)
        fail(KDSS_ERR_UNSUPPORTED, "in-place iterations exist for the integer rule only");
    const long double lim = st.precision == KDSS_INT64 ? 9.2e18L : 9.007199254740992e15L;
    const long double ck = (long double)st.ck_lo + (long double)st.ck_hi * 18446744073709551616.0L;
    if ((long double)(st.t + T) * ck >= lim)
        fail(KDSS_ERR_OVERFLOW, "T * c_k leaves the exact range of r");
    cudaGraphExec_t exec = nullptr;
    const long long nk = capture(c, &exec, [&](const Ctx &cc) {
        KDSS_CUDA(cudaMemsetAsync(st.ovf_count.p, 0, sizeof(int), cc.stream));
        if (st.precision == KDSS_FP64)
            launch_pbupdate_int<double>(cc, s, st.k, (double *)st.r.p, (double *)st.r.p,
                                        st.ovf_list.p, st.ovf_count.p, st.err.p);
        else
            launch_pbupdate_int<uint64_t>(cc, s, st.k, st.r.p, st.r.p, st.ovf_list.p,
                                          st.ovf_count.p, st.err.p);
    });
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < T && e == cudaSuccess; ++it) {
        e = cudaGraphLaunch(exec, c.stream);
        add_launches(nk);
    }
    cudaGraphExecDestroy(exec);
    check_cuda(e, "in-place FW graph launch", __FILE__, __LINE__);
    enqueue_step(c, s, st);  // delta is zero: only the max of r
    st.t += T;
}

// One in-place iteration's launches for a query of the server (slow-list
// reset and PBUpdate scattering into r itself); the server refreshes the max
// of r with a step over the zero delta before it extracts.
void fw_enqueue_inplace(const Ctx &c, const SctDev &s, StateDev &st) {
    if (st.precision == KDSS_FP32K)
        fail(KDSS_ERR_UNSUPPORTED, "in-place iterations exist for the integer rule only");
    KDSS_CUDA(cudaMemsetAsync(st.ovf_count.p, 0, sizeof(int), c.stream));
    if (st.precision == KDSS_FP64)
        launch_pbupdate_int<double>(c, s, st.k, (double *)st.r.p, (double *)st.r.p, st.ovf_list.p,
                                    st.ovf_count.p, st.err.p);
    else
        launch_pbupdate_int<uint64_t>(c, s, st.k, st.r.p, st.r.p, st.ovf_list.p, st.ovf_count.p,
                                      st.err.p);
}

// ---- several SCTs over disjoint node ranges sharing one state (batches) ----

void fw_init_n(const Ctx &c, int64_t n, int64_t short_capacity, int precision, StateDev &st) {
    SctDev shell;
    shell.n = n;
    shell.class_begin[0] = 0;
    shell.class_begin[3] = short_capacity;
    fw_init(c, shell, precision, st);
}

void fw_enqueue_group(const Ctx &c, const SctDev &s, StateDev &st, int64_t node_off, int k) {
    if (k < 0) k = s.k;
    // the slow-pair list is shared by the groups of one iteration
    KDSS_CUDA(cudaMemsetAsync(st.ovf_count.p, 0, sizeof(int), c.stream));
    if (st.precision == KDSS_FP32K) {
        launch_pbupdate_f32_on(c, s, k, st, st.r32.p + node_off, st.a32.p + node_off,
                               st.a32c.p + node_off);
    } else if (st.precision == KDSS_FP64) {
        launch_pbupdate_int<double>(c, s, k, (double *)st.r.p + node_off,
                                    (double *)st.acc.p + node_off, st.ovf_list.p, st.ovf_count.p,
                                    st.err.p);
    } else {
        launch_pbupdate_int<uint64_t>(c, s, k, st.r.p + node_off, st.acc.p + node_off,
                                      st.ovf_list.p, st.ovf_count.p, st.err.p);
    }
}

void fw_enqueue_step_range(const Ctx &c, StateDev &st, int64_t node_off, int64_t n, bool advance) {
    if (n <= 0) return;
    const int B = 256;
    const int sgrid = grid_for(c, n, B, 4);
    if (st.precision == KDSS_FP32K) {
        k_step_f32<<<sgrid, B, 0, c.stream>>>(n, st.r32.p + node_off, st.r32c.p + node_off,
                                             st.a32.p + node_off, st.a32c.p + node_off, st.dev_t.p,
                                             (unsigned int *)(st.dev_t.p + 1), st.ovf_count.p,
                                             advance ? 1 : 0);
    } else if (st.precision == KDSS_FP64) {
        k_step_int<double><<<sgrid, B, 0, c.stream>>>(n, (double *)st.r.p + node_off,
                                                      (double *)st.acc.p + node_off, st.maxr.p,
                                                      st.ovf_count.p);
    } else {
        k_step_int<uint64_t><<<sgrid, B, 0, c.stream>>>(n, st.r.p + node_off, st.acc.p + node_off,
                                                        st.maxr.p, st.ovf_count.p);
    }
    KDSS_LAUNCH_CHECK();
}

// ---- work-queue plans ----

void queue_plan(const Ctx &c, const std::vector<std::pair<const SctDev *, int64_t>> &sets, int chunk,
                int tpp, QueuePlan &qp, int k) {
    qp.chunk = std::max(1, chunk);
    qp.tpp = tpp == 8 ? 8 : 32;
    std::vector<QGroup> hg;
    std::vector<QItem> hi, hl[2];
    for (size_t g = 0; g < sets.size(); ++g) {
        const SctDev &s = *sets[g].first;
        QGroup d{};
        d.pair_off = s.pair_off.p;
        d.nodes = s.nodes.p;
        d.h = s.h.p;
        d.binom = s.binom.p;
        d.binomf = s.binomf.p;
        d.bcols = s.bcols();
        d.k = k >= 0 ? k : s.k;
        d.node_off = sets[g].second;
        d.short_end = s.class_begin[3];
        d.long_begin[0] = s.class_begin[3];
        d.long_end[0] = s.class_begin[4];
        d.long_begin[1] = s.class_begin[4];
        d.long_end[1] = s.class_begin[5];
        hg.push_back(d);
        const int64_t tiles = ceil_div(d.short_end, 32);
        for (int64_t t = 0; t < tiles; t += qp.chunk)
            hi.push_back(QItem{(int32_t)g, 0, t, (int32_t)std::min<int64_t>(qp.chunk, tiles - t), 0});
        for (int kind = 1; kind <= 2; ++kind) {
            const int64_t b = d.long_begin[kind - 1], e = d.long_end[kind - 1];
            const int64_t per = 8 * (int64_t)qp.chunk;
            for (int64_t q = b; q < e; q += per)
                hl[kind - 1].push_back(
                    QItem{(int32_t)g, kind, q, (int32_t)std::min<int64_t>(per, e - q), 0});
        }
    }
    qp.nitems = (int)hi.size();
    qp.nlong[0] = (int)hl[0].size();
    qp.nlong[1] = (int)hl[1].size();
    qp.groups = DBuf<QGroup>(c, std::max<size_t>(hg.size(), 1));
    qp.items = DBuf<QItem>(c, std::max<size_t>(hi.size() + hl[0].size() + hl[1].size(), 1));
    qp.cursor = DBuf<unsigned>(c, 3);
    if (!hg.empty()) to_device(c, qp.groups.p, hg.data(), hg.size());
    if (!hi.empty()) to_device(c, qp.items.p, hi.data(), hi.size());
    if (!hl[0].empty()) to_device(c, qp.items.p + hi.size(), hl[0].data(), hl[0].size());
    if (!hl[1].empty()) to_device(c, qp.items.p + hi.size() + hl[0].size(), hl[1].data(), hl[1].size());
    sync(c);
}

template <class RT>
void queue_launch_long(const Ctx &c, QueuePlan &qp, StateDev &st, RT *r, RT *acc) {
    const int64_t base1 = qp.nitems, base2 = qp.nitems + qp.nlong[0];
    auto go = [&](auto kern, int n, int64_t base, unsigned *cur) {
        if (n == 0) return;
        const int grid = (int)std::min<int64_t>(ceil_div(n, FW_THREADS / 32), (int64_t)c.num_sms * 4);
        kern<<<grid, FW_THREADS, 0, c.stream>>>(qp.groups.p, qp.items.p + base, n, cur, r, acc,
                                                st.err.p);
        KDSS_LAUNCH_CHECK();
    };
    if (qp.tpp == 8) go(k_pb_queue_long<RT, 8, 32>, qp.nlong[0], base1, qp.cursor.p + 1);
    else go(k_pb_queue_long<RT, 32, 8>, qp.nlong[0], base1, qp.cursor.p + 1);
    go(k_pb_queue_long<RT, 32, 32>, qp.nlong[1], base2, qp.cursor.p + 2);
}

void queue_enqueue_f32(const Ctx &c, QueuePlan &qp, StateDev &st) {
    const int64_t base1 = qp.nitems, base2 = qp.nitems + qp.nlong[0];
    auto go = [&](auto kern, int n, int64_t base, unsigned *cur) {
        if (n == 0) return;
        const int grid = (int)std::min<int64_t>(ceil_div(n, FW_THREADS / 32), (int64_t)c.num_sms * 4);
        kern<<<grid, FW_THREADS, 0, c.stream>>>(qp.groups.p, qp.items.p + base, n, cur, st.r32.p,
                                                st.a32.p, st.a32c.p, st.dev_t.p, st.err.p);
        KDSS_LAUNCH_CHECK();
    };
    if (qp.tpp == 8) go(k_pb_queue_long_f32<8, 32>, qp.nlong[0], base1, qp.cursor.p + 1);
    else go(k_pb_queue_long_f32<32, 8>, qp.nlong[0], base1, qp.cursor.p + 1);
    go(k_pb_queue_long_f32<32, 32>, qp.nlong[1], base2, qp.cursor.p + 2);
    if (qp.nitems == 0) return;
    const int grid = (int)std::min<int64_t>(ceil_div(qp.nitems, QW), (int64_t)c.num_sms * 6);
    k_pb_queue_f32<<<grid, QW * 32, 0, c.stream>>>(qp.groups.p, qp.items.p, qp.nitems, qp.cursor.p,
                                                    st.r32.p, st.a32.p, st.a32c.p, st.dev_t.p,
                                                    st.err.p);
    KDSS_LAUNCH_CHECK();
}

void queue_enqueue(const Ctx &c, QueuePlan &qp, StateDev &st) {
    if (qp.nitems + qp.nlong[0] + qp.nlong[1] == 0) return;
    KDSS_CUDA(cudaMemsetAsync(qp.cursor.p, 0, 3 * sizeof(unsigned), c.stream));
    if (st.precision == KDSS_FP32K) {
        queue_enqueue_f32(c, qp, st);
        return;
    }
    if (st.precision == KDSS_FP64)
        queue_launch_long<double>(c, qp, st, (double *)st.r.p, (double *)st.acc.p);
    else
        queue_launch_long<uint64_t>(c, qp, st, st.r.p, st.acc.p);
    if (qp.nitems == 0) return;
    const size_t smem = sizeof(QSmem);
    static thread_local int attr_dev = -1;
    if (attr_dev != c.device) {
        KDSS_CUDA(cudaFuncSetAttribute(k_pb_queue<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
        KDSS_CUDA(cudaFuncSetAttribute(k_pb_queue<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
        attr_dev = c.device;
    }
    const int grid = (int)std::min<int64_t>(ceil_div(qp.nitems, QW), (int64_t)c.num_sms * 4);
    if (st.precision == KDSS_FP64)
        k_pb_queue<double><<<grid, QW * 32, smem, c.stream>>>(qp.groups.p, qp.items.p, qp.nitems,
                                                             qp.cursor.p, (double *)st.r.p,
                                                             (double *)st.acc.p, st.err.p);
    else
        k_pb_queue<uint64_t><<<grid, QW * 32, smem, c.stream>>>(qp.groups.p, qp.items.p, qp.nitems,
                                                               qp.cursor.p, st.r.p, st.acc.p,
                                                               st.err.p);
    KDSS_LAUNCH_CHECK();
}

// The step of one iteration over the whole state, advancing its count.
void fw_step_advance(const Ctx &c, StateDev &st, int64_t n) {
    fw_enqueue_step_range(c, st, 0, n, true);
    st.t += 1;
}

long long fw_capture(const Ctx &c, cudaGraphExec_t *exec, const std::function<void(const Ctx &)> &fn) {
    return capture(c, exec, fn);
}

}  // namespace kdss


