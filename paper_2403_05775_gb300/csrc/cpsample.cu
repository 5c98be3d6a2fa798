// cpsample.cu -- CPSample (Sec. 5, Alg. 4) on the GPU: k-cliques sampled as
// k-color paths, Alg. 1 over the sampled set, and its densest prefix.
//
// Readings (the oracle states the same ones):
//  S1 greedy colouring, vertices by decreasing rank of the build order, each
//     taking the smallest colour no coloured neighbour has.  On the GPU it is
//     computed in rounds (Jones-Plassmann with the rank as priority): a vertex
//     takes its colour once every higher-ranked neighbour has one, which gives
//     exactly the sequential greedy colouring.
//  S2 a k-color path has strictly increasing colours; dp[v][i] counts those of
//     i vertices from v (uint64, overflow reported).
//  S3 sample j draws word j of SplitMix64 (Steele, Lea, Flood 2014) seeded
//     with `seed`; R = floor((x >> 11) * #paths / 2^53) is the rank of its
//     path in the order (start id, then adjacency order).
//  S4 the sampled cliques form a set (rows sorted, duplicates removed).
#include <algorithm>
#include <cstring>

#include "handles.cuh"

namespace kdss {

void extract_from_cliques(const Ctx &c, const StateDev &st, const int32_t *cl, int64_t count,
                          int k, kdss_result *out);

namespace {

constexpr unsigned FULLC = 0xffffffffu;
constexpr int CP_MAXK = 16;
constexpr int COL_BITS = 4096;  // colours a warp can rule out in its bitmap

// one round of the colouring in rank space: position i takes its colour when
// all its out-neighbours (higher positions) have theirs
__global__ void k_color_round(int64_t n, const int64_t *__restrict__ oo,
                              const int32_t *__restrict__ oa, int32_t *colr, int *remaining,
                              int *err) {
    __shared__ uint32_t bits[8][COL_BITS / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t *bm = bits[wib];
    for (int64_t i = warp; i < n; i += nw) {
        if (colr[i] >= 0) continue;  // uniform per warp
        const int64_t e0 = oo[i], e1 = oo[i + 1];
        bool ready = true;
        for (int64_t e = e0 + lane; e < e1; e += 32)
            if (*(volatile int32_t *)&colr[oa[e]] < 0) ready = false;
        if (!__all_sync(FULLC, ready)) {
            if (lane == 0) atomicAdd(remaining, 1);
            continue;
        }
        const int64_t deg = e1 - e0;  // the colour is at most deg
        if (deg + 1 > COL_BITS) {
            if (lane == 0) atomicOr(err, DERR_CAPACITY);
            continue;
        }
        const int words = (int)((deg + 1 + 31) / 32);
        for (int w = lane; w < words; w += 32) bm[w] = 0u;
        __syncwarp();
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t cc = colr[oa[e]];
            if (cc <= deg) atomicOr(&bm[cc >> 5], 1u << (cc & 31));
        }
        __syncwarp();
        int first = -1;
        for (int w0 = 0; w0 < words && first < 0; w0 += 32) {
            const int w = w0 + lane;
            const uint32_t free = w < words ? ~bm[w] : 0u;
            const unsigned has = __ballot_sync(FULLC, free != 0u);
            if (has) {
                const int src = __ffs(has) - 1;
                const uint32_t f = __shfl_sync(FULLC, free, src);
                first = (w0 + src) * 32 + __ffs(f) - 1;
            }
        }
        if (lane == 0) colr[i] = first;
        __syncwarp();
    }
}

__global__ void k_color_to_ids(int64_t n, const int32_t *vert, const int32_t *colr, int32_t *color,
                               int *maxc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        color[vert[i]] = colr[i];
        atomicMax(maxc, colr[i]);
    }
}

// dp[v * k + (i - 1)] from dp[w * k + (i - 2)] over higher-coloured neighbours
__global__ void k_dp_level(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                           const int32_t *__restrict__ color, int k, int i, uint64_t *dp, int *err) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (i == 1) { dp[v * k] = 1ull; continue; }
        const int cv = color[v];
        unsigned long long lo = 0, hi = 0;
        for (int64_t e = off[v]; e < off[v + 1]; ++e) {
            const int32_t w = adj[e];
            if (color[w] > cv) {
                const unsigned long long x = dp[(int64_t)w * k + (i - 2)];
                lo += x;
                hi += lo < x ? 1ull : 0ull;
            }
        }
        if (hi) atomicOr(err, DERR_OVERFLOW);
        dp[v * k + (i - 1)] = lo;
    }
}

__global__ void k_dp_last(int64_t n, const uint64_t *dp, int k, int64_t *last) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        last[v] = (int64_t)dp[v * k + (k - 1)];
}

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t index) {
    uint64_t z = seed + (index + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool adjacent(const int64_t *off, const int32_t *adj, int32_t a, int32_t b) {
    int64_t lo = off[a], hi = off[a + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t x = adj[mid];
        if (x == b) return true;
        if (x < b) lo = mid + 1; else hi = mid;
    }
    return false;
}

// one thread per sample: the path of rank R, and whether it is a clique
// (then written, ids ascending, to its row; flag[j] = 1)
__global__ void k_sample(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                         const int32_t *__restrict__ color, int k, const uint64_t *__restrict__ dp,
                         const int64_t *__restrict__ incl, uint64_t total, int64_t t, uint64_t seed,
                         int32_t *rows, int32_t *flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < t;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = splitmix64_at(seed, (uint64_t)j) >> 11;
        // R = floor(x * total / 2^53), x < 2^53: the 117-bit product shifted
        const uint64_t plo = x * total, phi = __umul64hi(x, total);
        uint64_t R = (phi << 11) | (plo >> 53);
        // start: the first v with incl[v] > R
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((uint64_t)incl[mid] > R) hi = mid; else lo = mid + 1;
        }
        int64_t v = lo;
        R -= (uint64_t)incl[v] - dp[v * k + (k - 1)];
        int32_t P[CP_MAXK];
        P[0] = (int32_t)v;
        for (int i = k - 1; i >= 1; --i) {
            const int cv = color[v];
            for (int64_t e = off[v]; e < off[v + 1]; ++e) {
                const int32_t w = adj[e];
                if (color[w] <= cv) continue;
                const uint64_t cnt = dp[(int64_t)w * k + (i - 1)];
                if (R < cnt) { v = w; break; }
                R -= cnt;
            }
            P[k - i] = (int32_t)v;
        }
        bool ok = true;
        for (int a = 0; a < k && ok; ++a)
            for (int b = a + 2; b < k && ok; ++b) ok = adjacent(off, adj, P[a], P[b]);
        flag[j] = ok ? 1 : 0;
        if (ok) {
            for (int a = 1; a < k; ++a) {  // ids ascending
                const int32_t y = P[a];
                int b = a - 1;
                while (b >= 0 && P[b] > y) { P[b + 1] = P[b]; --b; }
                P[b + 1] = y;
            }
            for (int a = 0; a < k; ++a) rows[(size_t)j * k + a] = P[a];
        }
    }
}

__global__ void k_flags_to_i64(int64_t t, const int32_t *flag, int64_t *f64) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < t;
         j += (int64_t)gridDim.x * blockDim.x)
        f64[j] = flag[j];
}

__global__ void k_compact_rows(int64_t t, const int32_t *flag, const int64_t *at, const int32_t *rows,
                               int k, int32_t *out) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < t;
         j += (int64_t)gridDim.x * blockDim.x)
        if (flag[j])
            for (int a = 0; a < k; ++a) out[(size_t)at[j] * k + a] = rows[(size_t)j * k + a];
}

__global__ void k_col_keys(int64_t c, const int32_t *rows, int k, int col, const int32_t *perm,
                           uint64_t *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint64_t)(uint32_t)rows[(size_t)perm[i] * k + col];
}

__global__ void k_iota(int64_t c, int32_t *p) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

__global__ void k_unique_rows(int64_t c, const int32_t *rows, int k, const int32_t *perm,
                              int64_t *first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool nw = i == 0;
        if (!nw)
            for (int a = 0; a < k; ++a)
                if (rows[(size_t)perm[i] * k + a] != rows[(size_t)perm[i - 1] * k + a]) { nw = true; break; }
        first[i] = nw ? 1 : 0;
    }
}

__global__ void k_gather_unique(int64_t c, const int32_t *rows, int k, const int32_t *perm,
                                const int64_t *first, const int64_t *at, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < c;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (first[i])
            for (int a = 0; a < k; ++a) out[(size_t)at[i] * k + a] = rows[(size_t)perm[i] * k + a];
    }
}

}  // namespace

void cpsample_run(const Ctx &c, const kdss_graph_desc &g, int k, int64_t t, int T, uint64_t seed,
                  int order, kdss_result *out, kdss_cpsample_stats *stats) {
    if (k < 2 || k > CP_MAXK) fail(KDSS_ERR_INVALID_ARG, "CPSample: k must be in [2, 16]");
    if (t < 0 || t > ((int64_t)1 << 31)) fail(KDSS_ERR_INVALID_ARG, "CPSample: t must be in [0, 2^31]");
    if (T < 0) fail(KDSS_ERR_INVALID_ARG, "T must be >= 0");
    memset(out, 0, sizeof *out);
    kdss_cpsample_stats stt{};
    GraphDev gd;
    build_graph(c, g, order, gd);
    const int64_t n = gd.n;
    const int B = 256;
    DBuf<int> ctl(c, 3);  // [0] remaining, [1] err, [2] max colour
    zero(c, ctl.p, 3 * sizeof(int));
    DBuf<int32_t> color(c, (size_t)std::max<int64_t>(n, 1));
    if (n > 0) {
        // S1: rounds of the colouring in rank space
        DBuf<int32_t> colr(c, (size_t)n);
        KDSS_CUDA(cudaMemsetAsync(colr.p, 0xff, (size_t)n * 4, c.stream));
        const int grid = grid_for(c, n * 32, B, 8);
        for (int64_t round = 0;; ++round) {
            if (round > n) fail(KDSS_ERR_CUDA, "CPSample colouring did not finish");
            zero(c, ctl.p, sizeof(int));
            k_color_round<<<grid, B, 0, c.stream>>>(n, gd.out_off.p, gd.out_adj.p, colr.p, ctl.p, ctl.p + 1);
            KDSS_LAUNCH_CHECK();
            int h[2] = {0, 0};
            to_host(c, h, ctl.p, 2);
            if (h[1]) fail(KDSS_ERR_UNSUPPORTED, "CPSample: a vertex with more than 4095 higher-ranked neighbours");
            if (h[0] == 0) break;
        }
        k_color_to_ids<<<grid_for(c, n, B), B, 0, c.stream>>>(n, gd.vert.p, colr.p, color.p, ctl.p + 2);
        KDSS_LAUNCH_CHECK();
        int mc = 0;
        to_host(c, &mc, ctl.p + 2, 1);
        stt.colors = mc + 1;
    }
    // S2: path counts
    DBuf<uint64_t> dp(c, (size_t)std::max<int64_t>(n * k, 1));
    for (int i = 1; i <= k && n > 0; ++i) {
        k_dp_level<<<grid_for(c, n, B), B, 0, c.stream>>>(n, gd.off.p, gd.adj.p, color.p, k, i, dp.p,
                                                          ctl.p + 1);
        KDSS_LAUNCH_CHECK();
    }
    DBuf<int64_t> last(c, (size_t)std::max<int64_t>(n, 1)), incl(c, (size_t)std::max<int64_t>(n, 1));
    uint64_t total = 0;
    if (n > 0) {
        int e = 0;
        to_host(c, &e, ctl.p + 1, 1);
        if (e) fail(KDSS_ERR_OVERFLOW, "CPSample: more than 2^64 color paths from a vertex");
        k_dp_last<<<grid_for(c, n, B), B, 0, c.stream>>>(n, dp.p, k, last.p);
        KDSS_LAUNCH_CHECK();
        // prefix sums of the per-vertex path counts: exact while n * max < 2^63
        const uint64_t mx = reduce_max_u64(c, (const uint64_t *)last.p, n);
        if (mx >= (1ull << 63) / (uint64_t)n)
            fail(KDSS_ERR_OVERFLOW, "CPSample: color-path counts too large for 63-bit prefix sums");
        inclusive_scan_u64_async(c, (const uint64_t *)last.p, (uint64_t *)incl.p, n);
        int64_t tot = 0;
        to_host(c, &tot, incl.p + (n - 1), 1);
        total = (uint64_t)tot;
    }
    stt.paths_total = total;
    stt.samples = t;
    // S3: samples; cliques among them
    DBuf<int32_t> set;
    int64_t nset = 0;
    if (t > 0 && total > 0) {
        DBuf<int32_t> rows(c, (size_t)t * k), flag(c, (size_t)t);
        k_sample<<<grid_for(c, t, B, 8), B, 0, c.stream>>>(n, gd.off.p, gd.adj.p, color.p, k, dp.p,
                                                           incl.p, total, t, seed, rows.p, flag.p);
        KDSS_LAUNCH_CHECK();
        DBuf<int64_t> f64(c, (size_t)t), at(c, (size_t)t);
        k_flags_to_i64<<<grid_for(c, t, B), B, 0, c.stream>>>(t, flag.p, f64.p);
        KDSS_LAUNCH_CHECK();
        const int64_t nc = exclusive_scan_i64(c, f64.p, at.p, t);
        stt.samples_clique = nc;
        if (nc > 0) {
            DBuf<int32_t> cl(c, (size_t)nc * k);
            k_compact_rows<<<grid_for(c, t, B), B, 0, c.stream>>>(t, flag.p, at.p, rows.p, k, cl.p);
            KDSS_LAUNCH_CHECK();
            rows.reset();
            // S4: rows in lexicographic order (LSD over the columns), duplicates out
            DBuf<int32_t> perm(c, (size_t)nc);
            DBuf<uint64_t> keys(c, (size_t)nc);
            k_iota<<<grid_for(c, nc, B), B, 0, c.stream>>>(nc, perm.p);
            KDSS_LAUNCH_CHECK();
            const int bits = bit_length((uint64_t)std::max<int64_t>(n, 1));
            for (int col = k - 1; col >= 0; --col) {
                k_col_keys<<<grid_for(c, nc, B), B, 0, c.stream>>>(nc, cl.p, k, col, perm.p, keys.p);
                KDSS_LAUNCH_CHECK();
                radix_sort_u64(c, keys.p, perm.p, nc, {{0, bits}});
            }
            DBuf<int64_t> first(c, (size_t)nc), pos(c, (size_t)nc);
            k_unique_rows<<<grid_for(c, nc, B), B, 0, c.stream>>>(nc, cl.p, k, perm.p, first.p);
            KDSS_LAUNCH_CHECK();
            nset = exclusive_scan_i64(c, first.p, pos.p, nc);
            set = DBuf<int32_t>(c, (size_t)nset * k);
            k_gather_unique<<<grid_for(c, nc, B), B, 0, c.stream>>>(nc, cl.p, k, perm.p, first.p, pos.p,
                                                                   set.p);
            KDSS_LAUNCH_CHECK();
        }
    }
    stt.cliques = nset;
    // Alg. 1 over the set, then the sampled-density prefix
    StateDev st;
    fw_init_n(c, n, 1, KDSS_INT64, st);
    fw_cliques_run(c, set.p, nset, k, st, T);
    extract_from_cliques(c, st, set.p, nset, k, out);
    out->T = T;
    out->status = KDSS_OK;
    sync(c);
    if (stats) *stats = stt;
}

}  // namespace kdss
