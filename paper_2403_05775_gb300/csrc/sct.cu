// sct.cu -- step A3: the succinct clique tree restricted to P_k.
//
// Sec. 2 and Lemmas 2.4-2.5: the pairs (V_h, V_p) of the SCT encode every
// clique exactly once as V_h plus a subset of V_p; P_k keeps the pairs with
// |V_h| <= k <= |V(P)|, whose k-cliques partition C_k(V).  The construction
// (cited by the paper from Pivoter) is a pivoting recursion per root vertex v
// over its later neighbours N+(v) in the build order:
//   node (cand, hold, pivot):
//     cand empty          -> emit (hold, pivot) when |hold| <= k <= |hold|+|pivot|
//     otherwise pick the candidate x with the most neighbours inside cand
//     (ties: earliest in the order);
//       pivot branch      (cand & N(x), hold, pivot + x)
//       for each w in cand \ N[x], in order:
//                          (cand & N(w), hold + w, pivot), then cand -= w
//   pruned when |hold| > k or |hold| + |pivot| + |cand| < k (Lemma 2.5).
//
// GPU mapping: one warp per root, roots handed out by an atomic counter.
// The root's out-neighbourhood (d <= max out-degree) becomes a d x d bitset
// adjacency matrix; the recursion is an explicit depth-first stack of
// candidate / to-do bitsets, one 32-bit word per lane.  A count pass sizes
// every (length class, root) slot, an exclusive scan turns the counts into
// offsets, and an emit pass re-runs the same recursion and writes the pairs.
#include <algorithm>
#include <cmath>

#include "sct.cuh"

namespace kdss {

namespace {
// Correctly rounded (to nearest, ties to even) float of a 128-bit integer.
float u128_to_float(U128 x) {
    if (x.hi == 0 && x.lo < (1ull << 24)) return (float)x.lo;
    const int nb = bit_length_u128(x);          // > 24
    const int sh = nb - 24;                      // bits dropped
    auto bit = [&](int i) -> unsigned { return i >= 64 ? (unsigned)((x.hi >> (i - 64)) & 1ull)
                                                       : (unsigned)((x.lo >> i) & 1ull); };
    unsigned long long m = 0;
    for (int i = nb - 1; i >= sh; --i) m = (m << 1) | bit(i);
    const unsigned half = bit(sh - 1);
    bool sticky = false;
    for (int i = sh - 2; i >= 0 && !sticky; --i) sticky = bit(i) != 0;
    if (half && (sticky || (m & 1ull))) ++m;     // may carry into bit 24
    return ldexpf((float)m, sh);                 // exact: m < 2^25
}
}  // namespace

BinomTables host_binom_tables(int rows, int k) {
    const int cols = k + 1;
    BinomTables t;
    t.t128.assign((size_t)rows * cols, U128(0));
    t.t64.assign((size_t)rows * cols, 0);
    t.tf.assign((size_t)rows * cols, 0.f);
    for (int a = 0; a < rows; ++a) {
        for (int b = 0; b <= k; ++b) {
            U128 v(0);
            if (b > a) v = U128(0);
            else if (b == 0 || b == a) v = U128(1);
            else {
                const U128 x = t.t128[(size_t)(a - 1) * cols + b - 1], y = t.t128[(size_t)(a - 1) * cols + b];
                if (x == U128_OVF || y == U128_OVF) v = U128_OVF;
                else {
                    v = x + y;
                    if (v.hi < x.hi || (v.hi == x.hi && v.lo < x.lo) || v == U128_OVF) v = U128_OVF;
                }
            }
            const size_t i = (size_t)a * cols + b;
            t.t128[i] = v;
            t.t64[i] = (v.hi == 0 && v.lo < (1ull << 63)) ? v.lo : ~0ull;
            t.tf[i] = v == U128_OVF ? INFINITY : u128_to_float(v);
        }
    }
    return t;
}

std::vector<uint64_t> host_binom_table(int rows, int k) { return host_binom_tables(rows, k).t64; }

namespace {

constexpr int SCT_THREADS = 256;
constexpr int SCT_WARPS = SCT_THREADS / 32;

__host__ __device__ inline size_t ws_words(int dmax, int S) {
    size_t f = (size_t)dmax + 2;
    return (size_t)dmax + (size_t)dmax * S + 2 * f * S + 6 * f;
}

__device__ __forceinline__ int dev_class(int len) {
    return len <= 8 ? 0 : len <= 16 ? 1 : len <= 32 ? 2 : len <= 256 ? 3 : len <= 1024 ? 4 : -1;
}

// A work item is a node of the recursion: level 0 items are the roots; a
// hold branch whose candidate set has at least SPLIT_MIN vertices (and whose
// hold set can still grow) becomes an item of the next level instead of being
// walked inline, so that dense regions are spread over many warps.  (On the
// 1e5-node power-law benchmark graph a whole SCT build takes 1.9 ms less with
// a threshold of 8 than of 16; 6 and 8 are equal, 24 is far slower.)
// Record of a spawned item (uint32 words): root, |hold|, hold[0..k) (local
// indices; the root is -1), candidate bitset [S], pivot bitset [S].
constexpr int SPLIT_MIN = 8;
enum { MODE_COUNT = 0, MODE_SPAWN = 1, MODE_EMIT = 2, MODE_TOTAL = 3 };

// Totals of a count-only pass (MODE_TOTAL): roots in a pseudo-random order,
// each walked to the end by one warp (no spawned items, nothing stored), until
// a deadline.  Class NCLASS counts pairs longer than the FW kernels take.
struct CountTotals {
    unsigned long long pairs[NCLASS + 1], nodes[NCLASS + 1];  // roots walked to the end
    unsigned long long ck[2];                                   // their c_k (lo, hi)
    unsigned long long roots_done, roots_cut;                   // finished / cut by the deadline
    unsigned long long cut_pairs, cut_nodes;                    // pairs seen in the cut roots
    int maxlen, cbits;
};

struct ItemsIn {
    int64_t nitems;
    const uint32_t *rec;     // nullptr: the items are the roots root_base + 0..nitems-1
    int stride;              // words per record
    int64_t root_base = 0;
};
struct PassOut {
    int64_t *cntP;           // [NCLASS * nitems] class-major (COUNT)
    int64_t *cntN;
    int64_t *nspawn;         // [nitems] (COUNT)
    unsigned long long *ck;  // [2] lo, hi (COUNT)
    uint32_t *direct_rec;            // spawn records written by the count pass (COUNT)
    unsigned long long *direct_cursor;
    long long direct_cap;
    unsigned long long *nodes_seen;  // node entries counted so far, all levels (COUNT)
    unsigned long long node_budget;  // more than this: stop counting (COUNT)
    int *stop;                       // set once the budget is exceeded (COUNT)
    int *maxlen;             // (COUNT)
    int *cbits;              // bit length of the largest n_C (COUNT)
    const int64_t *spawn_off;  // [nitems] (SPAWN)
    uint32_t *spawn_rec;       // (SPAWN)
    const int64_t *baseP;    // [NCLASS * nitems] output offsets (EMIT)
    const int64_t *baseN;
    int64_t *pair_off;
    int32_t *nodes;
    uint8_t *h;
    uint16_t *lidx;                  // root-shared form (EMIT)
    int32_t *proot;
    CountTotals *tot;                // (TOTAL)
    unsigned long long perm_mul;     // root of item i: (i * perm_mul) mod n (TOTAL)
    unsigned long long budget_ns;    // each warp stops this long after it started (TOTAL)
};

// WPL: candidate-bitset words per lane (a root's out-degree is at most
// 1024 * WPL - 1); word wi of a bitset belongs to lane wi % 32.
template <int MODE, int WPL>
__global__ void __launch_bounds__(SCT_THREADS)
k_sct(int64_t n, const int64_t *__restrict__ out_off, const int32_t *__restrict__ out_adj,
      const int32_t *__restrict__ vert, int k, int klo, int dmax, int S,
      const uint64_t *__restrict__ binom, const U128 *__restrict__ binom128, int bcols,
      uint32_t *gws, int use_shared, unsigned long long *next_item, ItemsIn items, PassOut po,
      int *err) {
    extern __shared__ uint32_t smem[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const size_t ww = ws_words(dmax, S);
    uint32_t *base = use_shared ? smem + (size_t)wib * ww : gws + (size_t)gwarp * ww;
    const int F = dmax + 2;
    int32_t *O = (int32_t *)base;
    uint32_t *A = base + dmax;
    uint32_t *cand = A + (size_t)dmax * S;
    uint32_t *todo = cand + (size_t)F * S;
    int32_t *hold = (int32_t *)(todo + (size_t)F * S);
    int32_t *piv = hold + F;
    int32_t *fnh = piv + F;
    int32_t *fnp = fnh + F;
    int32_t *fph = fnp + F;
    int32_t *ids = fph + F;
    const int64_t NI = items.nitems;
    const uint64_t t_start = MODE == MODE_TOTAL ? globaltimer_ns() : 0ull;

    while (true) {
        unsigned long long rr = 0;
        if (lane == 0) {
            // a count pass over budget stops handing out items, and so does a
            // count-only pass past its deadline
            if (MODE == MODE_COUNT && *(volatile int *)po.stop) rr = ~0ull;
            else if (MODE == MODE_TOTAL && globaltimer_ns() - t_start > po.budget_ns) rr = ~0ull;
            else rr = atomicAdd(next_item, 1ull);
        }
        rr = __shfl_sync(FULL, rr, 0);
        if (rr >= (unsigned long long)NI) break;
        // items are handed out last to first: the roots late in the build
        // order (the densest region, the longest recursions) start first and
        // the many short items fill in behind them; every pass maps the
        // counter to items the same way, so outputs keep their item slots
        const int64_t item = MODE == MODE_TOTAL ? (int64_t)rr : NI - 1 - (int64_t)rr;
        const uint32_t *rec = items.rec ? items.rec + (size_t)item * items.stride : nullptr;
        const int64_t root = rec ? (int64_t)rec[0]
                                 : (MODE == MODE_TOTAL ? (int64_t)(((unsigned long long)item * po.perm_mul) %
                                                                   (unsigned long long)n)
                                                       : items.root_base + item);
        const int64_t o0 = out_off[root];
        const int d = (int)(out_off[root + 1] - o0);
        if (!rec && d + 1 < klo) {   // no pair of this root has k nodes
            if (MODE == MODE_TOTAL && lane == 0) atomicAdd(&po.tot->roots_done, 1ull);
            continue;
        }
        const int W = (d + 31) >> 5;

        // local vertex list and its adjacency bitsets
        for (int j = lane; j < d; j += 32) O[j] = out_adj[o0 + j];
        for (int q = lane; q < d * S; q += 32) A[q] = 0u;
        __syncwarp();
        // one row per lane: the later neighbours of O[j] that are in O (both
        // lists ascending, so a merge), each edge set in both rows
        for (int j = lane; j < d; j += 32) {
            const int32_t u = O[j];
            int64_t e = out_off[u];
            const int64_t e1 = out_off[u + 1];
            int x = j + 1;  // later than u, so after j in O
            while (e < e1 && x < d) {
                const int32_t w = out_adj[e], ox = O[x];
                if (w < ox) ++e;
                else if (ox < w) ++x;
                else {
                    atomicOr(&A[(size_t)j * S + (x >> 5)], 1u << (x & 31));
                    atomicOr(&A[(size_t)x * S + (j >> 5)], 1u << (j & 31));
                    ++e;
                    ++x;
                }
            }
        }
        // per-item outputs (lane 0)
        int64_t cP[NCLASS + 1], cN[NCLASS + 1];
#pragma unroll
        for (int c = 0; c < NCLASS + 1; ++c) {
            cP[c] = (MODE == MODE_EMIT && c < NCLASS) ? po.baseP[(int64_t)c * NI + item] : 0;
            cN[c] = (MODE == MODE_EMIT && c < NCLASS) ? po.baseN[(int64_t)c * NI + item] : 0;
        }
        bool cut = false;            // TOTAL: the deadline stopped this root's walk
        unsigned steps = 0;
        int64_t nsp = MODE == MODE_SPAWN ? po.spawn_off[item] : 0;
        unsigned long long ck_lo = 0, ck_hi = 0;
        unsigned long long pend = 0;  // node entries not yet added to nodes_seen
        int mlen = 0;
        int cbits = 0;                // bit length of the largest n_C counted

        // initial frame: the root, or the spawned recursion node
        if (!rec) {
#pragma unroll
            for (int u = 0; u < WPL; ++u) {
                const int wi = lane + 32 * u;
                if (wi < W) {
                    const int rem = d - wi * 32;
                    cand[wi] = rem >= 32 ? FULL : ((1u << rem) - 1u);
                }
            }
            if (lane == 0) { fnh[0] = 1; fnp[0] = 0; fph[0] = 0; hold[0] = -1; }
        } else {
            const int nh0 = (int)rec[1];
            const uint32_t *rc = rec + 2 + k;
            const uint32_t *rp = rc + S;
#pragma unroll
            for (int u = 0; u < WPL; ++u)
                if (lane + 32 * u < W) cand[lane + 32 * u] = rc[lane + 32 * u];
            if (lane == 0) {
                for (int t = 0; t < nh0; ++t) hold[t] = (int32_t)rec[2 + t];
                int np0 = 0;
                for (int w = 0; w < W; ++w) {
                    uint32_t b = rp[w];
                    while (b) { piv[np0++] = w * 32 + __ffs(b) - 1; b &= b - 1; }
                }
                fnh[0] = nh0; fnp[0] = np0; fph[0] = 0;
            }
        }
        __syncwarp();
        int depth = 0;
        while (depth >= 0) {
            if (MODE == MODE_TOTAL && ((++steps) & 4095u) == 0u) {
                int late = 0;
                if (lane == 0) late = globaltimer_ns() - t_start > po.budget_ns ? 1 : 0;
                if (__shfl_sync(FULL, late, 0)) { cut = true; break; }
            }
            uint32_t *cd = cand + (size_t)depth * S;
            uint32_t *td = todo + (size_t)depth * S;
            const int h = fnh[depth], p = fnp[depth];
            if (fph[depth] == 0) {
                uint32_t cw[WPL];
                unsigned pc = 0;
#pragma unroll
                for (int u = 0; u < WPL; ++u) {
                    cw[u] = lane + 32 * u < W ? cd[lane + 32 * u] : 0u;
                    pc += (unsigned)__popc(cw[u]);
                }
                const int nc = (int)__reduce_add_sync(FULL, pc);
                if (h > k || h + p + nc < klo) { --depth; continue; }
                if (nc == 0) {
                    if (h <= k && klo <= h + p) {
                        const int len = h + p;
                        const int cls = dev_class(len);
                        // c_k of the hold cap k; a k-agnostic build (klo < k) keeps
                        // pairs with fewer than k nodes and ignores the count's range
                        const U128 nC = p >= k - h ? binom128[(size_t)p * bcols + (k - h)] : U128(0);
                        const bool ovf = nC == U128_OVF;
                        if (MODE == MODE_TOTAL) {
                            if (lane == 0) {
                                const int c6 = cls < 0 ? NCLASS : cls;
                                cP[c6] += 1;
                                cN[c6] += len;
                                mlen = len > mlen ? len : mlen;
                                if (ovf) {
                                    cbits = 129;
                                } else {
                                    unsigned long long o = ck_lo;
                                    ck_lo += nC.lo;
                                    ck_hi += nC.hi + (ck_lo < o ? 1ull : 0ull);
                                    const int nb = nC.hi ? 128 - __clzll((long long)nC.hi)
                                                         : 64 - __clzll((long long)nC.lo);
                                    cbits = nb > cbits ? nb : cbits;
                                }
                            }
                        } else if (cls < 0 || (klo == k && ovf)) {
                            if (lane == 0) atomicOr(err, cls < 0 ? DERR_CAPACITY : DERR_OVERFLOW);
                        } else if (MODE == MODE_COUNT) {
                            int over = 0;
                            if (lane == 0) {
                                cP[cls] += 1;
                                cN[cls] += len;
                                if (!ovf) {
                                    unsigned long long o = ck_lo;
                                    ck_lo += nC.lo;
                                    ck_hi += nC.hi + (ck_lo < o ? 1ull : 0ull);
                                    const int nb = nC.hi ? 128 - __clzll((long long)nC.hi)
                                                         : 64 - __clzll((long long)nC.lo);
                                    cbits = nb > cbits ? nb : cbits;
                                }
                                mlen = len > mlen ? len : mlen;
                                // report progress against the memory budget
                                // every 2^16 node entries, and stop once over
                                pend += (unsigned long long)len;
                                if (pend >= (1ull << 16)) {
                                    const unsigned long long t = atomicAdd(po.nodes_seen, pend) + pend;
                                    pend = 0;
                                    if (t > po.node_budget) atomicExch(po.stop, 1);
                                    over = *(volatile int *)po.stop;
                                }
                            }
                            if (__shfl_sync(FULL, over, 0)) break;
                        } else if (MODE == MODE_EMIT) {
                            int64_t pidx = 0, noff = 0;
                            if (lane == 0) {
                                pidx = cP[cls]++;
                                noff = cN[cls];
                                cN[cls] += len;
                            }
                            pidx = __shfl_sync(FULL, pidx, 0);
                            noff = __shfl_sync(FULL, noff, 0);
                            for (int t = lane; t < len; t += 32) {
                                int32_t id;
                                uint32_t flag;
                                if (t < h) {
                                    const int li = hold[t];
                                    id = li < 0 ? vert[root] : vert[O[li]];
                                    flag = HOLD_BIT;
                                } else {
                                    id = vert[O[piv[t - h]]];
                                    flag = 0u;
                                }
                                ids[t] = (int32_t)((uint32_t)id | flag);
                            }
                            __syncwarp();
                            for (int t = lane; t < len; t += 32) {
                                const int32_t raw = ids[t];
                                const int32_t my = raw & 0x7fffffff;
                                int pos = 0;
                                for (int u = 0; u < len; ++u) pos += ((ids[u] & 0x7fffffff) < my) ? 1 : 0;
                                po.nodes[noff + pos] = raw;
                                // the same node as an index into the root's
                                // neighbourhood (0 = the root), V_h mark in bit 15
                                const int li = t < h ? hold[t] : piv[t - h];
                                po.lidx[noff + pos] = (uint16_t)((li < 0 ? 0 : li + 1) | (t < h ? 0x8000 : 0));
                            }
                            if (lane == 0) {
                                po.pair_off[pidx] = noff;
                                po.h[pidx] = (uint8_t)h;
                                po.proot[pidx] = (int32_t)root;
                            }
                            __syncwarp();
                        }
                    }
                    --depth;
                    continue;
                }
                // pivot: most neighbours inside cand, smallest index on ties
                int bc = -1, bx = 0x7fffffff;
                for (int x = lane; x < d; x += 32) {
                    if ((cd[x >> 5] >> (x & 31)) & 1u) {
                        const uint32_t *ax = A + (size_t)x * S;
                        int cnt = 0;
                        for (int w = 0; w < W; ++w) cnt += __popc(ax[w] & cd[w]);
                        if (cnt > bc) { bc = cnt; bx = x; }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    int obc = __shfl_xor_sync(FULL, bc, o);
                    int obx = __shfl_xor_sync(FULL, bx, o);
                    if (obc > bc || (obc == bc && obx < bx)) { bc = obc; bx = obx; }
                }
                if (depth + 1 >= F) {  // cannot happen: each level adds a node
                    if (lane == 0) atomicOr(err, DERR_LOGIC);
                    break;
                }
                const uint32_t *ax = A + (size_t)bx * S;
#pragma unroll
                for (int u = 0; u < WPL; ++u) {
                    const int wi = lane + 32 * u;
                    if (wi < W) {
                        uint32_t tw = cw[u] & ~ax[wi];
                        if (wi == (bx >> 5)) tw &= ~(1u << (bx & 31));
                        if (h >= k) tw = 0u;  // hold branches would exceed k
                        td[wi] = tw;
                        cand[(size_t)(depth + 1) * S + wi] = cw[u] & ax[wi];
                    }
                }
                if (lane == 0) {
                    fph[depth] = 1;
                    piv[p] = bx;
                    fnh[depth + 1] = h;
                    fnp[depth + 1] = p + 1;
                    fph[depth + 1] = 0;
                }
                __syncwarp();
                ++depth;
            } else {
                // the first non-empty to-do word (lowest index)
                uint32_t tw[WPL];
                unsigned first = 0xffffffffu;
#pragma unroll
                for (int u = WPL - 1; u >= 0; --u) {
                    const int wi = lane + 32 * u;
                    tw[u] = wi < W ? td[wi] : 0u;
                    if (tw[u]) first = (unsigned)wi;
                }
                const unsigned src = __reduce_min_sync(FULL, first);
                if (src == 0xffffffffu) { --depth; continue; }
                uint32_t mine = tw[0];
#pragma unroll
                for (int u = 1; u < WPL; ++u)
                    if ((int)(src >> 5) == u) mine = tw[u];
                const uint32_t word = __shfl_sync(FULL, mine, src & 31);
                const int w = (int)src * 32 + __ffs(word) - 1;
                if (depth + 1 >= F) {
                    if (lane == 0) atomicOr(err, DERR_LOGIC);
                    break;
                }
                const uint32_t *aw = A + (size_t)w * S;
                uint32_t child[WPL];
                unsigned pcc = 0;
#pragma unroll
                for (int u = 0; u < WPL; ++u) {
                    const int wi = lane + 32 * u;
                    child[u] = 0u;
                    if (wi < W) {
                        const uint32_t c0 = cd[wi];
                        child[u] = c0 & aw[wi];
                        if (wi == (int)src) {
                            td[wi] = tw[u] & ~(1u << (w & 31));
                            cd[wi] = c0 & ~(1u << (w & 31));
                        }
                    }
                    pcc += (unsigned)__popc(child[u]);
                }
                const int ncc = (int)__reduce_add_sync(FULL, pcc);
                // big hold branch: becomes an item of the next level
                if (MODE != MODE_TOTAL && h + 1 < k && ncc >= SPLIT_MIN && h + 1 + p + ncc >= klo) {
                    // the count pass also writes the record, at a slot taken
                    // from a cursor, while the slots last; if they run out,
                    // a spawn pass writes every record in item order
                    uint32_t *r2 = nullptr;
                    if (MODE == MODE_COUNT) {
                        long long slot = 0;
                        if (lane == 0) slot = (long long)atomicAdd(po.direct_cursor, 1ull);
                        slot = __shfl_sync(FULL, slot, 0);
                        if (slot < po.direct_cap) r2 = po.direct_rec + (size_t)slot * (2 + k + 2 * S);
                        nsp += 1;
                    } else if (MODE == MODE_SPAWN) {
                        r2 = po.spawn_rec + (size_t)nsp * (2 + k + 2 * S);
                        nsp += 1;
                    }
                    if (r2) {
                        if (lane == 0) {
                            r2[0] = (uint32_t)root;
                            r2[1] = (uint32_t)(h + 1);
                            for (int t = 0; t < h; ++t) r2[2 + t] = (uint32_t)hold[t];
                            r2[2 + h] = (uint32_t)w;
                            for (int t = h + 1; t < k; ++t) r2[2 + t] = 0u;
                        }
#pragma unroll
                        for (int u = 0; u < WPL; ++u) {
                            const int wi = lane + 32 * u;
                            if (wi < S) {
                                r2[2 + k + wi] = wi < W ? child[u] : 0u;
                                uint32_t pw = 0u;
                                for (int t = 0; t < p; ++t)
                                    if ((piv[t] >> 5) == wi) pw |= 1u << (piv[t] & 31);
                                r2[2 + k + S + wi] = pw;
                            }
                        }
                    }
                    __syncwarp();
                    continue;  // stay at this depth: next hold branch
                }
#pragma unroll
                for (int u = 0; u < WPL; ++u)
                    if (lane + 32 * u < W) cand[(size_t)(depth + 1) * S + lane + 32 * u] = child[u];
                if (lane == 0) {
                    hold[h] = w;
                    fnh[depth + 1] = h + 1;
                    fnp[depth + 1] = p;
                    fph[depth + 1] = 0;
                }
                __syncwarp();
                ++depth;
            }
        }
        if (MODE == MODE_TOTAL && lane == 0) {
            CountTotals *T = po.tot;
            if (!cut) {
#pragma unroll
                for (int c = 0; c < NCLASS + 1; ++c) {
                    if (cP[c]) atomicAdd(&T->pairs[c], (unsigned long long)cP[c]);
                    if (cN[c]) atomicAdd(&T->nodes[c], (unsigned long long)cN[c]);
                }
                if (ck_lo || ck_hi) {
                    unsigned long long old = atomicAdd(&T->ck[0], ck_lo);
                    unsigned long long carry = (old + ck_lo < old) ? 1ull : 0ull;
                    if (ck_hi + carry) atomicAdd(&T->ck[1], ck_hi + carry);
                }
                atomicAdd(&T->roots_done, 1ull);
                atomicMax(&T->maxlen, mlen);
                atomicMax(&T->cbits, cbits);
            } else {
                unsigned long long pp = 0, nn = 0;
#pragma unroll
                for (int c = 0; c < NCLASS + 1; ++c) { pp += cP[c]; nn += cN[c]; }
                atomicAdd(&T->cut_pairs, pp);
                atomicAdd(&T->cut_nodes, nn);
                atomicAdd(&T->roots_cut, 1ull);
            }
        }
        if (MODE == MODE_COUNT && lane == 0) {
            if (pend) {
                const unsigned long long t = atomicAdd(po.nodes_seen, pend) + pend;
                if (t > po.node_budget) atomicExch(po.stop, 1);
                pend = 0;
            }
#pragma unroll
            for (int c = 0; c < NCLASS; ++c) {
                po.cntP[(int64_t)c * NI + item] = cP[c];
                po.cntN[(int64_t)c * NI + item] = cN[c];
            }
            po.nspawn[item] = nsp;
            if (ck_lo || ck_hi) {
                unsigned long long old = atomicAdd(&po.ck[0], ck_lo);
                unsigned long long carry = (old + ck_lo < old) ? 1ull : 0ull;
                if (ck_hi + carry) atomicAdd(&po.ck[1], ck_hi + carry);
            }
            atomicMax(po.maxlen, mlen);
            atomicMax(po.cbits, cbits);
        }
        __syncwarp();
    }
}

// ---- caller-given pairs -> device layout ---------------------------------
__global__ void k_pair_classes(int64_t np, const int64_t *off, const int32_t *h, int k,
                               int64_t n, const int32_t *nodes, uint64_t *keys, int *err) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t len = off[q + 1] - off[q];
        int cls = dev_class((int)(len > 2048 ? 2048 : len));
        if (len < 0 || cls < 0 || h[q] < 0 || h[q] > k || len < k) {
            atomicOr(err, DERR_BAD_ID);
            cls = NCLASS - 1;
        }
        keys[q] = ((uint64_t)cls << 32) | (uint64_t)q;
    }
    (void)n; (void)nodes;
}

__global__ void k_pair_lens(int64_t np, const uint64_t *keys, const int64_t *off, int64_t *lens) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = (int64_t)(keys[i] & 0xffffffffu);
        lens[i] = off[q + 1] - off[q];
    }
}

// warp per pair: copy with ids sorted ascending and the hold flag set
__global__ void k_pair_copy(int64_t np, const uint64_t *keys, const int64_t *off,
                            const int32_t *h, const int32_t *nodes, const int64_t *newoff,
                            int64_t n, int32_t *onodes, uint8_t *oh, int *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < np; i += nwarps) {
        const int64_t q = (int64_t)(keys[i] & 0xffffffffu);
        const int64_t b = off[q], len = off[q + 1] - b;
        const int hq = h[q];
        for (int64_t t = lane; t < len; t += 32) {
            const int32_t my = nodes[b + t];
            if (my < 0 || my >= n) { atomicOr(err, DERR_BAD_ID); continue; }
            int64_t pos = 0;
            for (int64_t u = 0; u < len; ++u) {
                int32_t o = nodes[b + u];
                pos += (o < my || (o == my && u < t)) ? 1 : 0;
            }
            onodes[newoff[i] + pos] = (int32_t)((uint32_t)my | (t < hq ? HOLD_BIT : 0u));
        }
        if (lane == 0) oh[i] = (uint8_t)hq;
    }
}

__global__ void k_pair_ck(int64_t np, const int64_t *off, const uint8_t *h, const U128 *binom128,
                          int bcols, int k, unsigned long long *ck, int *maxlen, int *cbits,
                          int *err) {
    unsigned long long lo = 0, hi = 0;
    int ml = 0, mb = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
         q += (int64_t)gridDim.x * blockDim.x) {
        int len = (int)(off[q + 1] - off[q]);
        int hq = h[q], p = len - hq;
        if (hq > k || len < k) continue;   // not in P_k (a k-agnostic SCT counted at k)
        const U128 nC = binom128[(size_t)p * bcols + (k - hq)];
        if (nC == U128_OVF) { atomicOr(err, DERR_OVERFLOW); continue; }
        unsigned long long o = lo;
        lo += nC.lo;
        hi += nC.hi + (lo < o ? 1ull : 0ull);
        const int nb = nC.hi ? 128 - __clzll((long long)nC.hi) : 64 - __clzll((long long)nC.lo);
        mb = nb > mb ? nb : mb;
        ml = len > ml ? len : ml;
    }
    unsigned long long old = atomicAdd(&ck[0], lo);
    unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
    if (hi + carry) atomicAdd(&ck[1], hi + carry);
    atomicMax(maxlen, ml);
    atomicMax(cbits, mb);
}

void upload_binom(const Ctx &c, int rows, int k, SctDev &out) {
    BinomTables t = host_binom_tables(rows, k);
    out.binom = DBuf<uint64_t>(c, t.t64.size());
    out.binom128 = DBuf<U128>(c, t.t128.size());
    out.binomf = DBuf<float>(c, t.tf.size());
    to_device(c, out.binom.p, t.t64.data(), t.t64.size());
    to_device(c, out.binom128.p, t.t128.data(), t.t128.size());
    to_device(c, out.binomf.p, t.tf.data(), t.tf.size());
    out.binom_rows = rows;
    sync(c);  // the host tables go out of scope
}

// c_k is a sum of eta counts below 2^cbits each: it fits 128 bits when
// cbits + bit_length(eta) <= 128.
void check_ck_range(int cbits, int64_t npairs) {
    if (cbits + bit_length((uint64_t)std::max<int64_t>(npairs, 1)) > 128)
        fail(KDSS_ERR_OVERFLOW, "c_k could need more than 128 bits");
}

}  // namespace

namespace {
// rnb_off[v] = out_off[v] + v; entry 0 of v's list is v's id, entry j + 1 the
// id of its j-th out-neighbour (rank space -> original ids).
__global__ void k_rnb(int64_t n, const int64_t *__restrict__ out_off, const int32_t *__restrict__ out_adj,
                      const int32_t *__restrict__ vert, int64_t *rnb_off, int32_t *rnb_ids) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nw) {
        const int64_t b = out_off[v], e = out_off[v + 1], o = b + v;
        if (lane == 0) {
            rnb_off[v] = o;
            rnb_ids[o] = vert[v];
            if (v == n - 1) rnb_off[n] = e + n;
        }
        for (int64_t j = b + lane; j < e; j += 32) rnb_ids[o + 1 + (j - b)] = vert[out_adj[j]];
    }
}
}  // namespace

void build_root_neighbourhoods(const Ctx &c, const GraphDev &g, SctDev &out) {
    const int64_t n = g.n;
    int64_t m1 = 0;
    if (n > 0) to_host(c, &m1, g.out_off.p + n, 1);
    out.rnb_off = DBuf<int64_t>(c, (size_t)n + 1);
    out.rnb_ids = DBuf<int32_t>(c, (size_t)std::max<int64_t>(n + m1, 1));
    if (n > 0) {
        const int B = 256;
        k_rnb<<<grid_for(c, n * 32, B), B, 0, c.stream>>>(n, g.out_off.p, g.out_adj.p, g.vert.p,
                                                          out.rnb_off.p, out.rnb_ids.p);
        KDSS_LAUNCH_CHECK();
    } else {
        zero(c, out.rnb_off.p, sizeof(int64_t));
    }
}

void build_sct(const Ctx &c, const GraphDev &g, int k, SctDev &out, int klo, int64_t root_lo,
               int64_t root_hi) {
    if (klo < 0) klo = k;
    const int64_t n = g.n;
    if (root_hi < 0) root_hi = n;
    root_lo = std::max<int64_t>(0, std::min<int64_t>(root_lo, n));
    root_hi = std::max<int64_t>(root_lo, std::min<int64_t>(root_hi, n));
    out.k = k;
    out.n = n;
    const int dmax = std::max(1, g.max_out);
    if (dmax + 1 > MAX_PAIR_LEN) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "out-degree %d above 1023 (degeneracy %d): pairs could exceed 1024 nodes",
                 g.max_out, g.degeneracy);
        fail(KDSS_ERR_UNSUPPORTED, buf);
    }
    const int S = (dmax + 31) / 32;
    upload_binom(c, dmax + 2, k, out);
    const int bcols = k + 1;
    const int stride = 2 + k + 2 * S;

    const size_t ww = ws_words(dmax, S);
    const size_t smem = ww * sizeof(uint32_t) * SCT_WARPS;
    int use_shared = smem <= 96 * 1024 ? 1 : 0;
    int grid;
    DBuf<uint32_t> gws;
    if (use_shared) {
        KDSS_CUDA(cudaFuncSetAttribute(k_sct<MODE_COUNT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        KDSS_CUDA(cudaFuncSetAttribute(k_sct<MODE_SPAWN, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        KDSS_CUDA(cudaFuncSetAttribute(k_sct<MODE_EMIT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        KDSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sct<MODE_COUNT, 1>, SCT_THREADS, smem));
        grid = c.num_sms * std::max(1, per_sm);
    } else {
        // global workspace: bound its size to about 1 GiB
        int64_t warps = std::max<int64_t>(SCT_WARPS, (int64_t)(1ull << 28) / (int64_t)ww);
        warps = std::min<int64_t>(warps, (int64_t)c.num_sms * 32);
        grid = (int)std::max<int64_t>(1, warps / SCT_WARPS);
        gws = DBuf<uint32_t>(c, (size_t)grid * SCT_WARPS * ww);
    }
    const size_t dyn = use_shared ? smem : 0;

    DBuf<unsigned long long> ctr(c, 4);  // [0] next item, [1..2] c_k, [3] node entries seen
    DBuf<int> ints(c, 4);                // [0] max len, [1] error, [2] over budget, [3] n_C bits
    zero(c, ctr.p, 4 * sizeof(unsigned long long));
    zero(c, ints.p, 4 * sizeof(int));
    // The SCT must fit the device: about 4.5 bytes per node entry (4 for the
    // id, the offset and h of pairs of ~20 nodes), within 85% of the free
    // memory at the start of the build.  The count pass stops once it has
    // seen more node entries than that.
    size_t free_b = 0, total_b = 0;
    KDSS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const unsigned long long node_budget = (unsigned long long)(0.85 * (double)free_b / 4.5);

    struct Level {
        int64_t nitems = 0;
        DBuf<uint32_t> rec;        // records (empty for the roots)
        DBuf<int64_t> cntP, cntN;  // [NCLASS * nitems]
    };
    std::vector<Level> levels;
    auto launch = [&](auto kern, const Level &L, const PassOut &po) {
        zero(c, ctr.p, sizeof(unsigned long long));
        int gsz = (int)std::min<int64_t>(grid, std::max<int64_t>(1, ceil_div(L.nitems, SCT_WARPS)));
        ItemsIn in{L.nitems, L.rec.p, stride, L.rec.p ? 0 : root_lo};
        kern<<<gsz, SCT_THREADS, dyn, c.stream>>>(n, g.out_off.p, g.out_adj.p, g.vert.p, k, klo, dmax,
                                                 S, out.binom.p, out.binom128.p, bcols, gws.p,
                                                 use_shared, ctr.p, in, po, ints.p + 1);
        KDSS_LAUNCH_CHECK();
    };
    // count and spawn, level by level; a spawned item has a larger hold set,
    // so there are at most k levels
    levels.reserve((size_t)k + 2);
    levels.emplace_back();
    levels[0].nitems = root_hi - root_lo;
    for (size_t lv = 0; lv < levels.size(); ++lv) {
        if (lv > (size_t)k) fail(KDSS_ERR_CUDA, "SCT build: more item levels than k");
        Level &L = levels[lv];
        if (L.nitems == 0) break;
        L.cntP = DBuf<int64_t>(c, (size_t)(NCLASS * L.nitems));
        L.cntN = DBuf<int64_t>(c, (size_t)(NCLASS * L.nitems));
        zero(c, L.cntP.p, L.cntP.bytes());  // items without pairs write nothing
        zero(c, L.cntN.p, L.cntN.bytes());
        DBuf<int64_t> nspawn(c, (size_t)L.nitems), spoff(c, (size_t)L.nitems);
        zero(c, nspawn.p, nspawn.bytes());
        // the count pass writes the next level's records into `direct` while
        // it has room (2 per item, at least 16384, at most 256 MB)
        const int64_t dcap = std::min<int64_t>(std::max<int64_t>(2 * L.nitems, 16384),
                                               (int64_t)(256ll << 20) / (4ll * stride));
        DBuf<uint32_t> direct(c, (size_t)dcap * stride);
        DBuf<unsigned long long> dcur(c, 1);
        zero(c, dcur.p, sizeof(unsigned long long));
        PassOut po{};
        po.cntP = L.cntP.p; po.cntN = L.cntN.p; po.nspawn = nspawn.p;
        po.ck = ctr.p + 1; po.maxlen = ints.p; po.cbits = ints.p + 3;
        po.nodes_seen = ctr.p + 3; po.node_budget = node_budget; po.stop = ints.p + 2;
        po.direct_rec = direct.p; po.direct_cursor = dcur.p; po.direct_cap = dcap;
        launch(k_sct<MODE_COUNT, 1>, L, po);
        {
            int over = 0;
            to_host(c, &over, ints.p + 2, 1);
            if (over) {
                unsigned long long seen = 0;
                to_host(c, &seen, ctr.p + 3, 1);
                char buf[320];
                snprintf(buf, sizeof buf,
                         "the SCT does not fit the device: the count pass stopped after %llu node "
                         "entries (about %.1f GB) with %.1f GB free; the SCT has more (k = %d, "
                         "degeneracy %d, out-degree %d)",
                         seen, 4.5e-9 * (double)seen, 1e-9 * (double)free_b, k, g.degeneracy,
                         g.max_out);
                fail(KDSS_ERR_OOM, buf);
            }
        }
        const int64_t ns = exclusive_scan_i64(c, nspawn.p, spoff.p, L.nitems);
        if (ns == 0) break;
        DBuf<uint32_t> rec;
        if (ns <= dcap) {
            rec = std::move(direct);  // every record is there (in arrival order)
        } else {
            direct.reset();
            rec = DBuf<uint32_t>(c, (size_t)ns * stride);
            PassOut ps{};
            ps.spawn_off = spoff.p;
            ps.spawn_rec = rec.p;
            launch(k_sct<MODE_SPAWN, 1>, L, ps);
        }
        levels.emplace_back();  // no reference into `levels` is used after this
        levels.back().nitems = ns;
        levels.back().rec = std::move(rec);
    }
    // output offsets: class-major over all items of all levels
    int64_t total = 0;
    for (auto &L : levels) {
        if (L.nitems > 0 && !L.cntP.p) fail(KDSS_ERR_CUDA, "SCT build: a level was not counted");
        total += L.nitems;
    }
    DBuf<int64_t> allP(c, (size_t)(NCLASS * std::max<int64_t>(total, 1)));
    DBuf<int64_t> allN(c, (size_t)(NCLASS * std::max<int64_t>(total, 1)));
    {
        int64_t b = 0;
        for (auto &L : levels) {
            if (!L.cntP.p) continue;
            for (int cl = 0; cl < NCLASS; ++cl) {
                KDSS_CUDA(cudaMemcpyAsync(allP.p + cl * total + b, L.cntP.p + cl * L.nitems,
                                          L.nitems * 8, cudaMemcpyDeviceToDevice, c.stream));
                KDSS_CUDA(cudaMemcpyAsync(allN.p + cl * total + b, L.cntN.p + cl * L.nitems,
                                          L.nitems * 8, cudaMemcpyDeviceToDevice, c.stream));
            }
            b += L.nitems;
        }
    }
    DBuf<int64_t> baseP(c, (size_t)(NCLASS * std::max<int64_t>(total, 1)));
    DBuf<int64_t> baseN(c, (size_t)(NCLASS * std::max<int64_t>(total, 1)));
    const int64_t npairs = exclusive_scan_i64(c, allP.p, baseP.p, NCLASS * total);
    const int64_t nnodes = exclusive_scan_i64(c, allN.p, baseN.p, NCLASS * total);
    unsigned long long hc[4];
    int hi[4];
    to_host(c, hc, ctr.p, 4);
    to_host(c, hi, ints.p, 4);
    if (hi[1] & DERR_OVERFLOW) fail(KDSS_ERR_OVERFLOW, "a pair's clique count needs more than 128 bits");
    if (hi[1] & DERR_CAPACITY) fail(KDSS_ERR_UNSUPPORTED, "a pair longer than 1024 nodes");
    if (hi[1]) fail(KDSS_ERR_CUDA, "SCT build: inconsistent device state");
    if (klo == k) check_ck_range(hi[3], npairs);
    out.ck_lo = hc[1];
    out.ck_hi = hc[2];
    out.max_len = hi[0];
    out.npairs = npairs;
    out.nnodes = nnodes;
    for (int cl = 0; cl < NCLASS; ++cl) {
        int64_t v = 0;
        if (total > 0) to_host(c, &v, baseP.p + (int64_t)cl * total, 1);
        out.class_begin[cl] = v;
    }
    out.class_begin[NCLASS] = npairs;
    allP.reset();
    allN.reset();
    out.pair_off = DBuf<int64_t>(c, (size_t)(npairs + 1));
    out.nodes = DBuf<int32_t>(c, (size_t)std::max<int64_t>(nnodes, 1) + NODES_PAD);
    out.h = DBuf<uint8_t>(c, (size_t)std::max<int64_t>(npairs, 1));
    out.proot = DBuf<int32_t>(c, (size_t)std::max<int64_t>(npairs, 1));
    out.lidx = DBuf<uint16_t>(c, (size_t)std::max<int64_t>(nnodes, 1) + NODES_PAD);
    build_root_neighbourhoods(c, g, out);
    if (npairs > 0) {
        // per-level slices of the class-major offsets
        int64_t b = 0;
        for (auto &L : levels) {
            if (!L.cntP.p) continue;
            DBuf<int64_t> lp(c, (size_t)(NCLASS * L.nitems)), ln(c, (size_t)(NCLASS * L.nitems));
            for (int cl = 0; cl < NCLASS; ++cl) {
                KDSS_CUDA(cudaMemcpyAsync(lp.p + cl * L.nitems, baseP.p + cl * total + b,
                                          L.nitems * 8, cudaMemcpyDeviceToDevice, c.stream));
                KDSS_CUDA(cudaMemcpyAsync(ln.p + cl * L.nitems, baseN.p + cl * total + b,
                                          L.nitems * 8, cudaMemcpyDeviceToDevice, c.stream));
            }
            PassOut pe{};
            pe.baseP = lp.p; pe.baseN = ln.p;
            pe.pair_off = out.pair_off.p; pe.nodes = out.nodes.p; pe.h = out.h.p;
            pe.lidx = out.lidx.p; pe.proot = out.proot.p;
            launch(k_sct<MODE_EMIT, 1>, L, pe);
            b += L.nitems;
        }
    }
    to_device(c, out.pair_off.p + npairs, &nnodes, 1);
    to_host(c, hi, ints.p, 2);
    if (hi[1]) fail(KDSS_ERR_CUDA, "SCT emit: inconsistent device state");
}

// Count-only pass: every root's recursion walked by one warp, nothing
// stored, so the sizes of an SCT far beyond the device can be measured.
// Roots are taken in the order i -> (i * P) mod n for a prime P that does
// not divide n (a permutation), so the roots finished before the deadline
// are a pseudo-random sample of all roots.
void sct_ck_at(const Ctx &c, const SctDev &s, int k, uint64_t &lo, uint64_t &hi) {
    if (k < 2 || k > s.k) fail(KDSS_ERR_INVALID_ARG, "k outside the range the SCT holds");
    const int B = 256;
    DBuf<unsigned long long> ck(c, 2);
    DBuf<int> ml(c, 3);
    zero(c, ck.p, 2 * sizeof(unsigned long long));
    zero(c, ml.p, 3 * sizeof(int));
    if (s.npairs > 0) {
        k_pair_ck<<<grid_for(c, s.npairs, B), B, 0, c.stream>>>(s.npairs, s.pair_off.p, s.h.p,
                                                               s.binom128.p, s.bcols(), k, ck.p,
                                                               ml.p, ml.p + 2, ml.p + 1);
        KDSS_LAUNCH_CHECK();
    }
    unsigned long long hc[2];
    int hm[3];
    to_host(c, hc, ck.p, 2);
    to_host(c, hm, ml.p, 3);
    if (hm[1] & DERR_OVERFLOW) fail(KDSS_ERR_OVERFLOW, "a pair's clique count needs more than 128 bits");
    check_ck_range(hm[2], s.npairs);
    lo = hc[0];
    hi = hc[1];
}

void count_sct(const Ctx &c, const GraphDev &g, int k, double budget_s, SctCount &out) {
    const int64_t n = g.n;
    out = SctCount{};
    out.roots_total = n;
    const int dmax = std::max(1, g.max_out);
    if (dmax > COUNT_MAX_OUT) {
        char buf[160];
        snprintf(buf, sizeof buf, "count-only pass: out-degree %d above %d", g.max_out, COUNT_MAX_OUT);
        fail(KDSS_ERR_UNSUPPORTED, buf);
    }
    if (n == 0) { out.complete = 1; return; }
    const int S = (dmax + 31) / 32;
    SctDev tab;
    upload_binom(c, dmax + 2, k, tab);
    const size_t ww = ws_words(dmax, S);
    const size_t smem = ww * sizeof(uint32_t) * SCT_WARPS;
    const int use_shared = smem <= 96 * 1024 ? 1 : 0;
    int grid;
    DBuf<uint32_t> gws;
    if (use_shared) {
        KDSS_CUDA(cudaFuncSetAttribute(k_sct<MODE_TOTAL, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        KDSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sct<MODE_TOTAL, 4>, SCT_THREADS, smem));
        grid = c.num_sms * std::max(1, per_sm);
    } else {
        // global workspace: a quarter of the free memory, at most 4 GiB
        size_t free_b = 0, total_b = 0;
        KDSS_CUDA(cudaMemGetInfo(&free_b, &total_b));
        const size_t cap = std::min<size_t>(free_b / 4, size_t(1) << 32);
        int64_t warps = (int64_t)(cap / (ww * sizeof(uint32_t)));
        warps = std::min<int64_t>(warps, (int64_t)c.num_sms * 32);
        if (warps < SCT_WARPS) fail(KDSS_ERR_OOM, "count-only pass: no room for one block's workspace");
        grid = (int)(warps / SCT_WARPS);
        gws = DBuf<uint32_t>(c, (size_t)grid * SCT_WARPS * ww);
    }
    grid = (int)std::min<int64_t>(grid, std::max<int64_t>(1, ceil_div(n, SCT_WARPS)));
    const size_t dyn = use_shared ? smem : 0;
    DBuf<CountTotals> tot(c, 1);
    DBuf<unsigned long long> next(c, 1);
    DBuf<int> err(c, 1);
    zero(c, tot.p, sizeof(CountTotals));
    zero(c, next.p, sizeof(unsigned long long));
    zero(c, err.p, sizeof(int));
    unsigned long long mul = 0;
    for (unsigned long long cand : {2654435761ull, 2246822519ull, 3266489917ull})
        if ((unsigned long long)n % cand != 0) { mul = cand % (unsigned long long)n; break; }
    if (mul == 0) mul = 1;
    PassOut po{};
    po.tot = tot.p;
    po.perm_mul = mul;
    po.budget_ns = budget_s <= 0 ? ~0ull : (unsigned long long)(budget_s * 1e9);
    ItemsIn in{n, nullptr, 0};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KDSS_CUDA(cudaEventCreate(&e0));
    KDSS_CUDA(cudaEventCreate(&e1));
    KDSS_CUDA(cudaEventRecord(e0, c.stream));
    k_sct<MODE_TOTAL, 4><<<grid, SCT_THREADS, dyn, c.stream>>>(n, g.out_off.p, g.out_adj.p, g.vert.p, k, k,
                                                           dmax, S, tab.binom.p, tab.binom128.p, k + 1,
                                                           gws.p, use_shared, next.p, in, po, err.p);
    KDSS_LAUNCH_CHECK();
    KDSS_CUDA(cudaEventRecord(e1, c.stream));
    CountTotals h;
    int he = 0;
    to_host(c, &h, tot.p, 1);
    to_host(c, &he, err.p, 1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (he) fail(KDSS_ERR_CUDA, "count-only pass: inconsistent device state");
    for (int cl = 0; cl <= NCLASS; ++cl) {
        out.pairs_per_class[cl] = (int64_t)h.pairs[cl];
        out.eta += (int64_t)h.pairs[cl];
        out.L += (int64_t)h.nodes[cl];
    }
    out.ck_lo = h.ck[0];
    out.ck_hi = h.ck[1];
    out.roots_done = (int64_t)h.roots_done;
    out.roots_cut = (int64_t)h.roots_cut;
    out.cut_pairs = (int64_t)h.cut_pairs;
    out.cut_nodes = (int64_t)h.cut_nodes;
    out.max_len = h.maxlen;
    out.count_bits = h.cbits;
    out.seconds = ms / 1e3;
    out.complete = (out.roots_done == n) ? 1 : 0;
}

void sct_from_pairs(const Ctx &c, int64_t n, int k, int64_t np, const int64_t *pair_off,
                    const int32_t *nodes, const int32_t *h, SctDev &out) {
    out.k = k;
    out.n = n;
    out.npairs = np;
    const int B = 256;
    DBuf<int> err(c, 1);
    zero(c, err.p, sizeof(int));
    DBuf<uint64_t> keys(c, (size_t)std::max<int64_t>(np, 1));
    if (np > 0) {
        k_pair_classes<<<grid_for(c, np, B), B, 0, c.stream>>>(np, pair_off, h, k, n, nodes, keys.p, err.p);
        KDSS_LAUNCH_CHECK();
    }
    int he = 0;
    to_host(c, &he, err.p, 1);
    if (he) fail(KDSS_ERR_INVALID_ARG, "pairs need 0 <= h <= k <= |V(P)| <= 1024");
    radix_sort_u64(c, keys.p, nullptr, np, {{32, 35}});
    DBuf<int64_t> lens(c, (size_t)std::max<int64_t>(np, 1));
    out.pair_off = DBuf<int64_t>(c, (size_t)(np + 1));
    int64_t nnodes = 0;
    if (np > 0) {
        k_pair_lens<<<grid_for(c, np, B), B, 0, c.stream>>>(np, keys.p, pair_off, lens.p);
        KDSS_LAUNCH_CHECK();
        nnodes = exclusive_scan_i64(c, lens.p, out.pair_off.p, np);
    }
    to_device(c, out.pair_off.p + np, &nnodes, 1);
    out.nnodes = nnodes;
    out.nodes = DBuf<int32_t>(c, (size_t)std::max<int64_t>(nnodes, 1) + NODES_PAD);
    out.h = DBuf<uint8_t>(c, (size_t)std::max<int64_t>(np, 1));
    if (np > 0) {
        k_pair_copy<<<grid_for(c, np * 32, B), B, 0, c.stream>>>(np, keys.p, pair_off, h, nodes,
                                                               out.pair_off.p, n, out.nodes.p,
                                                               out.h.p, err.p);
        KDSS_LAUNCH_CHECK();
    }
    // class boundaries from the sorted keys
    std::vector<uint64_t> hk((size_t)np);
    if (np > 0) to_host(c, hk.data(), keys.p, (size_t)np);
    for (int cl = 0; cl <= NCLASS; ++cl) {
        int64_t lo = 0, hi = np;
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if ((int)(hk[(size_t)mid] >> 32) < cl) lo = mid + 1; else hi = mid;
        }
        out.class_begin[cl] = lo;
    }
    out.class_begin[NCLASS] = np;
    // binomial table up to the longest pair, then c_k
    int maxlen = 0;
    if (np > 0) {
        std::vector<int64_t> hl((size_t)np);
        to_host(c, hl.data(), lens.p, (size_t)np);
        for (int64_t v : hl) maxlen = std::max<int>(maxlen, (int)v);
    }
    upload_binom(c, maxlen + 2, k, out);
    DBuf<unsigned long long> ck(c, 2);
    DBuf<int> ml(c, 2);
    zero(c, ck.p, 2 * sizeof(unsigned long long));
    zero(c, ml.p, 2 * sizeof(int));
    if (np > 0) {
        k_pair_ck<<<grid_for(c, np, B), B, 0, c.stream>>>(np, out.pair_off.p, out.h.p,
                                                         out.binom128.p, k + 1, k, ck.p, ml.p,
                                                         ml.p + 1, err.p);
        KDSS_LAUNCH_CHECK();
    }
    unsigned long long hc[2];
    int hm[2];
    to_host(c, hc, ck.p, 2);
    to_host(c, hm, ml.p, 2);
    to_host(c, &he, err.p, 1);
    if (he & DERR_BAD_ID) fail(KDSS_ERR_INVALID_ARG, "a pair node id is outside [0, n)");
    if (he & DERR_OVERFLOW) fail(KDSS_ERR_OVERFLOW, "a pair's clique count needs more than 128 bits");
    check_ck_range(hm[1], np);
    out.ck_lo = hc[0];
    out.ck_hi = hc[1];
    out.max_len = maxlen;
}

namespace {
__global__ void k_keep_flags(int64_t np, const int64_t *off, const uint8_t *h, int k, int64_t *keep,
                             int64_t *klen) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = off[q + 1] - off[q];
        const bool in = (int)h[q] <= k && (int64_t)k <= len;
        keep[q] = in ? 1 : 0;
        klen[q] = in ? len : 0;
    }
}

// warp per kept pair: nodes (ids ascending, hold bit kept) and h to their new place
__global__ void k_keep_copy(int64_t np, const int64_t *off, const int32_t *nodes, const uint8_t *h,
                            const int64_t *keep, const int64_t *pidx, const int64_t *noff,
                            int64_t *ooff, int32_t *onodes, uint8_t *oh) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = warp; q < np; q += nw) {
        if (!keep[q]) continue;
        const int64_t b = off[q], len = off[q + 1] - b, o = noff[q];
        for (int64_t t = lane; t < len; t += 32) onodes[o + t] = nodes[b + t];
        if (lane == 0) {
            ooff[pidx[q]] = o;
            oh[pidx[q]] = h[q];
        }
    }
}
}  // namespace

void sct_restrict(const Ctx &c, const SctDev &all, int k, SctDev &out) {
    const int64_t np = all.npairs;
    out.k = k;
    out.n = all.n;
    const int B = 256;
    DBuf<int64_t> keep(c, (size_t)std::max<int64_t>(np, 1)), klen(c, (size_t)std::max<int64_t>(np, 1));
    DBuf<int64_t> pidx(c, (size_t)std::max<int64_t>(np, 1)), noff(c, (size_t)std::max<int64_t>(np, 1));
    int64_t kept = 0, nn = 0;
    if (np > 0) {
        k_keep_flags<<<grid_for(c, np, B), B, 0, c.stream>>>(np, all.pair_off.p, all.h.p, k, keep.p, klen.p);
        KDSS_LAUNCH_CHECK();
        kept = exclusive_scan_i64(c, keep.p, pidx.p, np);
        nn = exclusive_scan_i64(c, klen.p, noff.p, np);
    }
    out.npairs = kept;
    out.nnodes = nn;
    out.pair_off = DBuf<int64_t>(c, (size_t)kept + 1);
    out.nodes = DBuf<int32_t>(c, (size_t)std::max<int64_t>(nn, 1) + NODES_PAD);
    out.h = DBuf<uint8_t>(c, (size_t)std::max<int64_t>(kept, 1));
    if (kept > 0) {
        k_keep_copy<<<grid_for(c, np * 32, B), B, 0, c.stream>>>(np, all.pair_off.p, all.nodes.p, all.h.p,
                                                               keep.p, pidx.p, noff.p, out.pair_off.p,
                                                               out.nodes.p, out.h.p);
        KDSS_LAUNCH_CHECK();
    }
    to_device(c, out.pair_off.p + kept, &nn, 1);
    // class boundaries: kept pairs before each boundary of the source
    for (int cl = 0; cl < NCLASS; ++cl) {
        const int64_t b = all.class_begin[cl];
        int64_t v = kept;
        if (b < np) to_host(c, &v, pidx.p + b, 1);
        out.class_begin[cl] = v;
    }
    out.class_begin[NCLASS] = kept;
    // binomials for k, then c_k and the longest pair
    upload_binom(c, std::max(all.max_len, 1) + 2, k, out);
    DBuf<unsigned long long> ck(c, 2);
    DBuf<int> ml(c, 3);
    zero(c, ck.p, 2 * sizeof(unsigned long long));
    zero(c, ml.p, 3 * sizeof(int));
    if (kept > 0) {
        k_pair_ck<<<grid_for(c, kept, B), B, 0, c.stream>>>(kept, out.pair_off.p, out.h.p,
                                                           out.binom128.p, k + 1, k, ck.p, ml.p,
                                                           ml.p + 2, ml.p + 1);
        KDSS_LAUNCH_CHECK();
    }
    unsigned long long hc[2];
    int hm[3];
    to_host(c, hc, ck.p, 2);
    to_host(c, hm, ml.p, 3);
    if (hm[1] & DERR_OVERFLOW) fail(KDSS_ERR_OVERFLOW, "a pair's clique count needs more than 128 bits");
    check_ck_range(hm[2], kept);
    out.ck_lo = hc[0];
    out.ck_hi = hc[1];
    out.max_len = hm[0];
}

}  // namespace kdss
