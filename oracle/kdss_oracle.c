/*
 * kdss_oracle.c -- plain, slow, single-threaded CPU oracle for PSCTL
 * (k-clique densest subgraph search by Frank-Wolfe over the succinct clique
 * tree; arxiv 2403.05775).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA solver shares
 * no code, header, table or helper with it.
 *
 * Every function cites the passage of the paper it restates.  Where the paper
 * is silent or ambiguous the reading taken is stated at the function.
 * Integers are exact (uint64 / unsigned __int128); the continuous rule works
 * in double (FP64).
 *
 * Readings of the paper used here:
 *  R1  Pairs in one FW iteration read the ranking of the previous iteration
 *      (synchronous / Jacobi form of Alg. 2); the in-place sequential form of
 *      Alg. 2 is provided as well (orc_fw_seq).
 *  R2  Alg. 3 hands the units left after the last whole round (fewer than
 *      the plateau's size) to randomly chosen nodes of the current plateau;
 *      here they go to the lowest original vertex ids
 *      (this reproduces Example 3.1, where the single clique of
 *      ({u4},{u5,u6}) goes to u4).
 *  R3  r starts at zero (Alg. 2 leaves the initial r open; Example 3.1
 *      starts from zeros).
 *  R4  The final sort of Alg. 2 is by non-increasing r, ties by ascending
 *      id.
 *  R5  Ties in the final argmax take the largest prefix (maximality of the
 *      k-clique densest subgraph, Def. 2.1).
 *  R6  Alg. 3 removes a node whose cap is used up only after an allocation
 *      round; nodes whose cap is zero from the start (every V_p node when
 *      |V_h| = k) are removed before the first round, otherwise the
 *      remainder units could go to them and exceed the C4 cap.
 *  R7  The SCT construction is only cited ([PIVOTER]).  It is restated from
 *      Lemmas 2.4-2.5: root v in the chosen vertex order with candidates
 *      N+(v); pivot = candidate with most neighbours among the candidates,
 *      ties to the earliest in the order; the pivot branch keeps the pivot as
 *      a "pivot" node, every non-neighbour w of the pivot (in order) opens a
 *      "hold" branch over the candidates adjacent to w that were not handled
 *      before; the k-pruning of Lemma 2.5 is applied during the recursion.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_BAD_GRAPH (-2)
#define ORC_OVERFLOW (-4)
#define ORC_OOM (-3)

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Binomial coefficients C(a, b); C(a, b) = 0 for b < 0 or b > a.           */
/* Lemma 2.6 counts the k-cliques of a pair and of each node with them.     */
/* Computed by the multiplicative formula in 128-bit (each partial product */
/* C(a-b+i, i) is an integer); *ovf is set when a value needs more than 64  */
/* bits.                                                                    */
/* ------------------------------------------------------------------------ */
/* *ovf128 (may be NULL) is set when a partial product would leave 128 bits. */
static u128 binom128_chk(int64_t a, int64_t b, int *ovf128) {
    if (b < 0 || a < 0 || b > a) return 0;
    if (b > a - b) b = a - b;
    u128 v = 1;
    for (int64_t i = 1; i <= b; ++i) {
        /* v * (a - b + i) / i = C(a - b + i, i) is an integer at every step;
           dividing v and i by their gcd first leaves i' dividing the factor,
           so the product overflows only when the value itself does */
        u128 f = (u128)(a - b + i), x = v, y = (u128)i;
        while (y) { const u128 t = x % y; x = y; y = t; }
        v /= x;
        f /= (u128)i / x;
        if (f && v > ~(u128)0 / f) { if (ovf128) *ovf128 = 1; return ~(u128)0; }
        v *= f;
    }
    return v;
}
static u128 binom128(int64_t a, int64_t b) { return binom128_chk(a, b, NULL); }

uint64_t orc_binom(int64_t a, int64_t b, int *ovf) {
    u128 v = binom128(a, b);
    if (v >> 64) { if (ovf) *ovf = 1; return UINT64_MAX; }
    return (uint64_t)v;
}

/* C(a, b) in 128 bits as (lo, hi); returns 1 when it needs more. */
int orc_binom128(int64_t a, int64_t b, uint64_t *lo, uint64_t *hi) {
    int o = 0;
    const u128 v = binom128_chk(a, b, &o);
    *lo = (uint64_t)v;
    *hi = (uint64_t)(v >> 64);
    return o;
}

/* ------------------------------------------------------------------------ */
/* A1: the simple undirected graph G(V, E) of Sec. 2 from a raw edge list.   */
/* Self-loops are dropped, both orientations kept, duplicates removed;       */
/* neighbour lists sorted by id.                                             */
/* ------------------------------------------------------------------------ */
static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

int orc_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
            int64_t **off_out, int32_t **adj_out, int64_t *nadj_out) {
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    if (!keys) return ORC_OOM;
    int64_t c = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t u = src[e], v = dst[e];
        if (u < 0 || v < 0 || u >= n || v >= n) { free(keys); return ORC_BAD_GRAPH; }
        if (u == v) continue;
        keys[c++] = ((uint64_t)u << 32) | (uint64_t)v;
        keys[c++] = ((uint64_t)v << 32) | (uint64_t)u;
    }
    qsort(keys, (size_t)c, sizeof(uint64_t), cmp_u64);
    int64_t uc = 0;
    for (int64_t i = 0; i < c; ++i)
        if (i == 0 || keys[i] != keys[i - 1]) keys[uc++] = keys[i];
    int64_t *off = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(uc + 1));
    for (int64_t i = 0; i < uc; ++i) {
        off[(keys[i] >> 32) + 1]++;
        adj[i] = (int32_t)(keys[i] & 0xffffffffu);
    }
    for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    free(keys);
    *off_out = off; *adj_out = adj; *nadj_out = uc;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* A2: degeneracy (Sec. 2: the smallest d such that every subgraph has a    */
/* vertex of degree <= d) by peeling.  Round form: at the current level c,   */
/* every remaining vertex of remaining degree <= c is removed in one round;  */
/* when none is left at level c, c rises to the smallest remaining degree.   */
/* core[v] = level at removal, round[v] = index of the removal round.        */
/* Returns the degeneracy (max core).                                        */
/* ------------------------------------------------------------------------ */
int64_t orc_peel(int64_t n, const int64_t *off, const int32_t *adj,
                 int32_t *core, int32_t *round_out) {
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    char *alive = (char *)malloc((size_t)n + 1);
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    for (int64_t v = 0; v < n; ++v) { deg[v] = off[v + 1] - off[v]; alive[v] = 1; }
    int64_t removed = 0, c = 0, rnd = 0, maxcore = 0;
    while (removed < n) {
        int64_t ns = 0;
        for (int64_t v = 0; v < n; ++v)
            if (alive[v] && deg[v] <= c) S[ns++] = (int32_t)v;
        if (ns == 0) {
            int64_t mn = INT64_MAX;
            for (int64_t v = 0; v < n; ++v)
                if (alive[v] && deg[v] < mn) mn = deg[v];
            c = mn;
            continue;
        }
        for (int64_t i = 0; i < ns; ++i) {
            alive[S[i]] = 0; core[S[i]] = (int32_t)c; round_out[S[i]] = (int32_t)rnd;
        }
        for (int64_t i = 0; i < ns; ++i) {
            int32_t v = S[i];
            for (int64_t e = off[v]; e < off[v + 1]; ++e)
                if (alive[adj[e]]) deg[adj[e]]--;
        }
        if (c > maxcore) maxcore = c;
        removed += ns;
        rnd++;
    }
    free(deg); free(alive); free(S);
    return maxcore;
}

/* Vertex order used by the SCT.  kind 0: key (peel round, id) -- a          */
/* degeneracy order, every vertex has at most core(v) later neighbours.      */
/* kind 1: key (core number, id).  rank[v] = position of v, vert[i] = vertex */
/* at position i.                                                            */
static const int32_t *g_key1;
static int cmp_key(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_key1[x] != g_key1[y]) return g_key1[x] < g_key1[y] ? -1 : 1;
    return x < y ? -1 : x > y;
}

void orc_order(int64_t n, const int32_t *core, const int32_t *round_, int kind,
               int32_t *rank, int32_t *vert) {
    for (int64_t i = 0; i < n; ++i) vert[i] = (int32_t)i;
    g_key1 = kind == 0 ? round_ : core;
    qsort(vert, (size_t)n, sizeof(int32_t), cmp_key);
    for (int64_t i = 0; i < n; ++i) rank[vert[i]] = (int32_t)i;
}

/* ------------------------------------------------------------------------ */
/* O1: explicit k-clique listing (definition of C_k(S), Sec. 2).  Cliques   */
/* are listed as increasing id sequences by extending with common           */
/* neighbours of larger id.  Output: c x k ids, or only the count when      */
/* out == NULL.  Returns the count, or -1 when it exceeds limit.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int64_t *off; const int32_t *adj; int k;
    int32_t *cur; int64_t count, cap, limit; int32_t **out;
} clq_ctx;

static int is_adj(const int64_t *off, const int32_t *adj, int32_t a, int32_t b) {
    int64_t lo = off[a], hi = off[a + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (adj[mid] < b) lo = mid + 1; else hi = mid;
    }
    return lo < off[a + 1] && adj[lo] == b;
}

static int clq_rec(clq_ctx *c, int depth, const int32_t *cand, int64_t nc) {
    if (depth == c->k) {
        if (c->limit >= 0 && c->count >= c->limit) return -1;
        if (c->out) {
            if (c->count >= c->cap) {
                c->cap = c->cap ? c->cap * 2 : 1024;
                *c->out = (int32_t *)realloc(*c->out, sizeof(int32_t) * (size_t)(c->cap * c->k));
            }
            memcpy(*c->out + c->count * c->k, c->cur, sizeof(int32_t) * (size_t)c->k);
        }
        c->count++;
        return 0;
    }
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc + 1));
    for (int64_t i = 0; i < nc; ++i) {
        int32_t v = cand[i];
        int64_t nn = 0;
        for (int64_t j = i + 1; j < nc; ++j)
            if (is_adj(c->off, c->adj, v, cand[j])) next[nn++] = cand[j];
        if (nn < c->k - depth - 1) continue;
        c->cur[depth] = v;
        if (clq_rec(c, depth + 1, next, nn) < 0) { free(next); return -1; }
    }
    free(next);
    return 0;
}

int64_t orc_list_cliques(int64_t n, const int64_t *off, const int32_t *adj, int k,
                         int64_t limit, int32_t **out) {
    clq_ctx c; memset(&c, 0, sizeof c);
    c.off = off; c.adj = adj; c.k = k; c.limit = limit; c.out = out;
    if (out) *out = NULL;
    c.cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(k + 1));
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    for (int64_t v = 0; v < n && c.count >= 0; ++v) {
        int64_t nc = 0;
        for (int64_t e = off[v]; e < off[v + 1]; ++e)
            if (adj[e] > v) cand[nc++] = adj[e];
        if (nc < k - 1) continue;
        c.cur[0] = (int32_t)v;
        if (k == 1) { /* single nodes */
            if (out) { if (c.count >= c.cap) { c.cap = c.cap ? c.cap * 2 : 1024;
                *out = (int32_t *)realloc(*out, sizeof(int32_t) * (size_t)c.cap); }
                (*out)[c.count] = (int32_t)v; }
            c.count++; continue;
        }
        if (clq_rec(&c, 1, cand, nc) < 0) { c.count = -1; break; }
    }
    free(cand); free(c.cur);
    return c.count;
}

/* ------------------------------------------------------------------------ */
/* O2: the SCT restricted to P_k (Sec. 2, Lemmas 2.4-2.5; reading R7).      */
/* Works in rank space: vertex i is vert[i]; adjacency is tested on the     */
/* original ids.  Pairs are emitted in root order, then depth-first order   */
/* (pivot branch first, then the hold branches in vertex order).  Nodes of a */
/* pair are written as original ids: V_h in the order added, then V_p in    */
/* the order added.                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const int64_t *off; const int32_t *adj; const int32_t *vert; int k;
    int64_t npairs, cap_pairs, nnodes, cap_nodes;
    int64_t *pair_off; int32_t *nodes; int32_t *hcnt;
    int count_only;
} sct_ctx;

static void sct_emit(sct_ctx *c, const int32_t *hold, int nh, const int32_t *piv, int np) {
    if (!c->count_only) {
        if (c->npairs + 1 >= c->cap_pairs) {
            c->cap_pairs = c->cap_pairs ? c->cap_pairs * 2 : 1024;
            c->pair_off = (int64_t *)realloc(c->pair_off, sizeof(int64_t) * (size_t)(c->cap_pairs + 1));
            c->hcnt = (int32_t *)realloc(c->hcnt, sizeof(int32_t) * (size_t)c->cap_pairs);
        }
        if (c->nnodes + nh + np >= c->cap_nodes) {
            c->cap_nodes = (c->cap_nodes ? c->cap_nodes * 2 : 4096) + nh + np;
            c->nodes = (int32_t *)realloc(c->nodes, sizeof(int32_t) * (size_t)c->cap_nodes);
        }
        c->pair_off[c->npairs] = c->nnodes;
        for (int i = 0; i < nh; ++i) c->nodes[c->nnodes + i] = c->vert[hold[i]];
        for (int i = 0; i < np; ++i) c->nodes[c->nnodes + nh + i] = c->vert[piv[i]];
        c->hcnt[c->npairs] = nh;
        c->pair_off[c->npairs + 1] = c->nnodes + nh + np;
    }
    c->nnodes += nh + np;
    c->npairs++;
}

static int radj(sct_ctx *c, int32_t a, int32_t b) {
    return is_adj(c->off, c->adj, c->vert[a], c->vert[b]);
}

static void sct_rec(sct_ctx *c, const int32_t *cand, int nc, int32_t *hold, int nh,
                    int32_t *piv, int np) {
    /* Lemma 2.5: no k-clique below this node. */
    if (nh > c->k) return;
    if (nh + np + nc < c->k) return;
    if (nc == 0) {
        if (nh <= c->k && c->k <= nh + np) sct_emit(c, hold, nh, piv, np);
        return;
    }
    /* pivot: most neighbours among the candidates, earliest on ties */
    int best = 0, bestc = -1;
    for (int i = 0; i < nc; ++i) {
        int cnt = 0;
        for (int j = 0; j < nc; ++j)
            if (j != i && radj(c, cand[i], cand[j])) cnt++;
        if (cnt > bestc) { bestc = cnt; best = i; }
    }
    int32_t x = cand[best];
    int32_t *sub = (int32_t *)calloc((size_t)(nc + 1), sizeof(int32_t));
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nc + 1));
    memcpy(cur, cand, sizeof(int32_t) * (size_t)nc);
    int ncur = nc;
    /* pivot branch: cliques inside N[x] -- x is optional (a pivot node) */
    int ns = 0;
    for (int j = 0; j < nc; ++j)
        if (cand[j] != x && radj(c, x, cand[j])) sub[ns++] = cand[j];
    piv[np] = x;
    sct_rec(c, sub, ns, hold, nh, piv, np + 1);
    /* hold branches: every candidate w outside N[x], in order; w is removed  */
    /* from the candidates once its branch is done                           */
    for (int i = 0; i < nc; ++i) {
        int32_t w = cand[i];
        if (w == x || radj(c, x, w)) continue;
        ns = 0;
        for (int j = 0; j < ncur; ++j)
            if (cur[j] != w && radj(c, w, cur[j])) sub[ns++] = cur[j];
        hold[nh] = w;
        sct_rec(c, sub, ns, hold, nh + 1, piv, np);
        int q = 0;
        for (int j = 0; j < ncur; ++j) if (cur[j] != w) cur[q++] = cur[j];
        ncur = q;
    }
    free(sub); free(cur);
}

/* rank/vert from orc_order.  Returns the number of pairs; arrays malloc'd. */
int64_t orc_sct(int64_t n, const int64_t *off, const int32_t *adj,
                const int32_t *rank, const int32_t *vert, int k, int count_only,
                int64_t **pair_off, int32_t **nodes, int32_t **hcnt, int64_t *nnodes) {
    sct_ctx c; memset(&c, 0, sizeof c);
    c.off = off; c.adj = adj; c.vert = vert; c.k = k; c.count_only = count_only;
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; ++v) if (off[v + 1] - off[v] > maxdeg) maxdeg = off[v + 1] - off[v];
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxdeg + 1));
    int32_t *hold = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxdeg + 2));
    int32_t *piv = (int32_t *)malloc(sizeof(int32_t) * (size_t)(maxdeg + 2));
    for (int64_t i = 0; i < n; ++i) {
        int32_t v = vert[i];
        int nc = 0;
        for (int64_t e = off[v]; e < off[v + 1]; ++e)
            if (rank[adj[e]] > i) cand[nc++] = rank[adj[e]];
        /* candidates in rank order */
        for (int a = 1; a < nc; ++a) {
            int32_t t = cand[a]; int b = a - 1;
            while (b >= 0 && cand[b] > t) { cand[b + 1] = cand[b]; --b; }
            cand[b + 1] = t;
        }
        hold[0] = (int32_t)i;
        sct_rec(&c, cand, nc, hold, 1, piv, 0);
    }
    free(cand); free(hold); free(piv);
    if (!count_only) {
        if (!c.pair_off) { c.pair_off = (int64_t *)calloc(1, sizeof(int64_t)); }
        c.pair_off[c.npairs] = c.nnodes;
        *pair_off = c.pair_off; *nodes = c.nodes; *hcnt = c.hcnt;
    }
    *nnodes = c.nnodes;
    return c.npairs;
}

/* ------------------------------------------------------------------------ */
/* PBUpdate (Alg. 3), integer form, reading R2 + R6.                         */
/* Input: the len nodes of a pair (original ids), their rankings r, h =     */
/* |V_h| (the first h nodes are V_h), k.  Output: delta[i] added to node i. */
/* The steps follow Alg. 3: the count n_C and the per-node upper bounds    */
/* (Lemma 2.6), plateaus of equal r in ascending order, then the walk that  */
/* raises the lowest plateau round by round.                                */
/* ------------------------------------------------------------------------ */
/* comparator inputs, one set per host thread (orc_fw_sync_par runs PBUpdate on several) */
static _Thread_local const uint64_t *g_sort_r; static _Thread_local const int32_t *g_sort_id;
static int cmp_by_r_id(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    if (g_sort_r[x] != g_sort_r[y]) return g_sort_r[x] < g_sort_r[y] ? -1 : 1;
    return g_sort_id[x] < g_sort_id[y] ? -1 : g_sort_id[x] > g_sort_id[y];
}
static int cmp_by_id(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return g_sort_id[x] < g_sort_id[y] ? -1 : g_sort_id[x] > g_sort_id[y];
}

int orc_pbupdate_alg3(int len, const int32_t *ids, const uint64_t *r_in, int h, int k,
                      uint64_t *delta) {
    int p = len - h;
    int ovf = 0;
    uint64_t nC = orc_binom(p, k - h, &ovf);                 /* cliques of the pair */
    uint64_t up_h = orc_binom(p, k - h, &ovf);               /* cap of a hold node */
    uint64_t up_p = orc_binom(p - 1, k - h - 1, &ovf);       /* cap of a pivot node */
    if (ovf) return ORC_OVERFLOW;
    uint64_t *r = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)len);
    uint64_t *up = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)len);
    int *srt = (int *)malloc(sizeof(int) * (size_t)len);
    int *A = (int *)malloc(sizeof(int) * (size_t)len);
    for (int i = 0; i < len; ++i) { r[i] = r_in[i]; up[i] = i < h ? up_h : up_p; }
    /* order by r; R6: nodes without capacity take no part */
    int ns = 0;
    for (int i = 0; i < len; ++i) if (up[i] > 0) srt[ns++] = i;
    g_sort_r = r_in; g_sort_id = ids;
    qsort(srt, (size_t)ns, sizeof(int), cmp_by_r_id);
    /* plateau boundaries: distinct levels r_1 < r_2 < ... < r_s */
    int *pstart = (int *)malloc(sizeof(int) * (size_t)(ns + 1));
    int s = 0;
    for (int j = 0; j < ns; ++j)
        if (j == 0 || r_in[srt[j]] != r_in[srt[j - 1]]) pstart[s++] = j;
    pstart[s] = ns;
    /* A holds V_i (the current plateau, with the merged lower plateaus) */
    int na = 0;
    int i = 0;                                               /* lowest plateau */
    while (nC > 0 && i < s) {                                /* units left to give */
        for (int j = pstart[i]; j < pstart[i + 1]; ++j) A[na++] = srt[j];
        uint64_t gap = (i + 1 >= s) ? UINT64_MAX
                       : r_in[srt[pstart[i + 1]]] - r_in[srt[pstart[i]]];   /* distance to the next level */
        while (nC > 0 && gap > 0 && na > 0) {                /* rounds on this plateau */
            uint64_t mu = UINT64_MAX;
            for (int j = 0; j < na; ++j) if (up[A[j]] < mu) mu = up[A[j]];
            uint64_t w = mu;                                 /* round size: min(cap, gap, n_C / |A|) */
            if (gap < w) w = gap;
            if (nC / (uint64_t)na < w) w = nC / (uint64_t)na;
            if (w > 0) {                                     /* w units to every node of A */
                for (int j = 0; j < na; ++j) { r[A[j]] += w; up[A[j]] -= w; }
                nC -= w * (uint64_t)na;
                if (gap != UINT64_MAX) gap -= w;
            } else {                                         /* fewer units than nodes (R2) */
                g_sort_id = ids;
                qsort(A, (size_t)na, sizeof(int), cmp_by_id);
                for (uint64_t j = 0; j < nC; ++j) { r[A[j]] += 1; up[A[j]] -= 1; }
                nC = 0;
            }
            int q = 0;                                       /* drop the capped nodes */
            for (int j = 0; j < na; ++j) if (up[A[j]] > 0) A[q++] = A[j];
            na = q;
        }
        /* what is left of the plateau joins the next one (kept in A) */
        i++;
    }
    int rc = nC == 0 ? ORC_OK : ORC_OVERFLOW;
    for (int j = 0; j < len; ++j) delta[j] = r[j] - r_in[j];
    free(r); free(up); free(srt); free(A); free(pstart);
    return rc;
}

/* The same allocation defined one clique at a time (the FW-2 step of Sec. 2 */
/* applied to each of the n_C cliques of the pair): each unit goes to the    */
/* node of smallest (r, id) that still has capacity.  Used to pin Alg. 3.    */
int orc_pbupdate_greedy(int len, const int32_t *ids, const uint64_t *r_in, int h, int k,
                        uint64_t *delta) {
    int p = len - h, ovf = 0;
    uint64_t nC = orc_binom(p, k - h, &ovf);
    uint64_t up_h = orc_binom(p, k - h, &ovf), up_p = orc_binom(p - 1, k - h - 1, &ovf);
    if (ovf) return ORC_OVERFLOW;
    uint64_t *r = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)len);
    uint64_t *up = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)len);
    for (int i = 0; i < len; ++i) { r[i] = r_in[i]; up[i] = i < h ? up_h : up_p; }
    for (uint64_t unit = 0; unit < nC; ++unit) {
        int b = -1;
        for (int i = 0; i < len; ++i) {
            if (up[i] == 0) continue;
            if (b < 0 || r[i] < r[b] || (r[i] == r[b] && ids[i] < ids[b])) b = i;
        }
        if (b < 0) { free(r); free(up); return ORC_OVERFLOW; }
        r[b]++; up[b]--;
    }
    for (int i = 0; i < len; ++i) delta[i] = r[i] - r_in[i];
    free(r); free(up);
    return ORC_OK;
}

/* Closed form of the same allocation: with g(L) = sum_u min(up_u,          */
/* max(0, L - r_u)), L is the largest integer with g(L) <= n_C; every node   */
/* gets min(up_u, max(0, L - r_u)) and the n_C - g(L) lowest ids among the   */
/* nodes with r_u <= L < r_u + up_u get one more.  Used to pin Alg. 3.       */
static u128 level_g(int len, const uint64_t *r, const uint64_t *up, u128 L) {
    u128 g = 0;
    for (int i = 0; i < len; ++i) {
        if ((u128)r[i] >= L) continue;
        u128 d = L - (u128)r[i];
        g += d < (u128)up[i] ? d : (u128)up[i];
    }
    return g;
}

int orc_pbupdate_level(int len, const int32_t *ids, const uint64_t *r, int h, int k,
                       uint64_t *delta) {
    int p = len - h, ovf = 0;
    uint64_t nC = orc_binom(p, k - h, &ovf);
    uint64_t up_h = orc_binom(p, k - h, &ovf), up_p = orc_binom(p - 1, k - h - 1, &ovf);
    if (ovf) return ORC_OVERFLOW;
    uint64_t *up = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)len);
    for (int i = 0; i < len; ++i) up[i] = i < h ? up_h : up_p;
    u128 lo = (u128)UINT64_MAX, hi = 0;
    for (int i = 0; i < len; ++i) {
        if ((u128)r[i] < lo) lo = r[i];
        if ((u128)r[i] + up[i] > hi) hi = (u128)r[i] + up[i];
    }
    /* g(lo) = 0 <= nC; g(hi) = k nC > nC (k >= 2): binary search */
    while (hi - lo > 1) {
        u128 mid = lo + (hi - lo) / 2;
        if (level_g(len, r, up, mid) <= nC) lo = mid; else hi = mid;
    }
    u128 L = lo;
    u128 g = level_g(len, r, up, L);
    uint64_t R = (uint64_t)((u128)nC - g);
    for (int i = 0; i < len; ++i) {
        u128 d = (u128)r[i] >= L ? 0 : L - r[i];
        delta[i] = (uint64_t)(d < up[i] ? d : up[i]);
    }
    while (R > 0) {
        int b = -1;
        for (int i = 0; i < len; ++i) {
            if (!((u128)r[i] <= L && L < (u128)r[i] + up[i])) continue;
            if ((u128)r[i] + delta[i] != L) continue;   /* already given the extra unit */
            if (b < 0 || ids[i] < ids[b]) b = i;
        }
        if (b < 0) { free(up); return ORC_OVERFLOW; }
        delta[b] += 1; R--;
    }
    free(up);
    return ORC_OK;
}

/* Continuous analogue of Alg. 3 (no floor: w = min(up, gap, n_C/|V_i|) as a */
/* real number), FP64.  The allocation is the exact water level of the pair. */
static _Thread_local const double *g_sort_rd;
static int cmp_by_rd_id(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    if (g_sort_rd[x] != g_sort_rd[y]) return g_sort_rd[x] < g_sort_rd[y] ? -1 : 1;
    return g_sort_id[x] < g_sort_id[y] ? -1 : g_sort_id[x] > g_sort_id[y];
}

int orc_pbupdate_cont(int len, const int32_t *ids, const double *r_in, int h, int k,
                      double *delta) {
    /* counts beyond 64 bits (long pairs, large k) are taken exactly in 128
       bits and rounded to double once (reading R10: exact binomials of
       Lemma 2.6 wherever they fit 128 bits) */
    int p = len - h, ovf = 0;
    double nC = (double)binom128_chk(p, k - h, &ovf);
    double up_h = nC, up_p = (double)binom128_chk(p - 1, k - h - 1, &ovf);
    if (ovf) return ORC_OVERFLOW;
    double *r = (double *)malloc(sizeof(double) * (size_t)len);
    double *up = (double *)malloc(sizeof(double) * (size_t)len);
    int *srt = (int *)malloc(sizeof(int) * (size_t)len);
    int *A = (int *)malloc(sizeof(int) * (size_t)len);
    int *pstart = (int *)malloc(sizeof(int) * (size_t)(len + 1));
    for (int i = 0; i < len; ++i) { r[i] = r_in[i]; up[i] = i < h ? up_h : up_p; }
    int ns = 0;
    for (int i = 0; i < len; ++i) if (up[i] > 0) srt[ns++] = i;
    g_sort_rd = r_in; g_sort_id = ids;
    qsort(srt, (size_t)ns, sizeof(int), cmp_by_rd_id);
    int s = 0;
    for (int j = 0; j < ns; ++j)
        if (j == 0 || r_in[srt[j]] != r_in[srt[j - 1]]) pstart[s++] = j;
    pstart[s] = ns;
    /* A: the current plateau V_i (lower plateaus merged in); all of its    */
    /* members sit at level lev.                                           */
    int na = 0, i = 0;
    while (nC > 0 && i < s) {
        for (int j = pstart[i]; j < pstart[i + 1]; ++j) A[na++] = srt[j];
        double lev = r_in[srt[pstart[i]]];
        double next = (i + 1 >= s) ? INFINITY : r_in[srt[pstart[i + 1]]];
        while (nC > 0 && lev < next && na > 0) {
            double mu = INFINITY;
            for (int j = 0; j < na; ++j) if (up[A[j]] < mu) mu = up[A[j]];
            double share = nC / (double)na, gap = next - lev;
            double w = mu < gap ? mu : gap;
            int last = share <= w;
            if (last) w = share;
            if (last) nC = 0; else nC -= w * (double)na;
            lev = (!last && w == gap) ? next : lev + w;
            for (int j = 0; j < na; ++j) { r[A[j]] = lev; up[A[j]] -= w; }
            int q = 0;                                   /* capped nodes leave */
            for (int j = 0; j < na; ++j) if (up[A[j]] > 0) A[q++] = A[j];
            na = q;
        }
        i++;
    }
    for (int j = 0; j < len; ++j) delta[j] = r[j] - r_in[j];
    free(r); free(up); free(srt); free(A); free(pstart);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* O3: PSCTL (Alg. 2) over a list of pairs.                                 */
/* ------------------------------------------------------------------------ */
static int max_pair_len(int64_t npairs, const int64_t *pair_off) {
    int64_t mx = 0;
    for (int64_t q = 0; q < npairs; ++q)
        if (pair_off[q + 1] - pair_off[q] > mx) mx = pair_off[q + 1] - pair_off[q];
    return (int)mx;
}

/* Synchronous iterations (R1): all pairs of iteration t read r_{t-1}. */
int orc_fw_sync(int64_t n, int64_t npairs, const int64_t *pair_off, const int32_t *nodes,
                const int32_t *hcnt, int k, int T, uint64_t *r) {
    int mx = max_pair_len(npairs, pair_off);
    uint64_t *dr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    uint64_t *rv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mx + 1));
    uint64_t *dv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mx + 1));
    int rc = ORC_OK;
    for (int t = 1; t <= T && rc == ORC_OK; ++t) {
        memset(dr, 0, sizeof(uint64_t) * (size_t)n);
        for (int64_t q = 0; q < npairs; ++q) {
            int len = (int)(pair_off[q + 1] - pair_off[q]);
            const int32_t *ids = nodes + pair_off[q];
            for (int i = 0; i < len; ++i) rv[i] = r[ids[i]];
            rc = orc_pbupdate_alg3(len, ids, rv, hcnt[q], k, dv);
            if (rc) break;
            for (int i = 0; i < len; ++i) dr[ids[i]] += dv[i];
        }
        for (int64_t v = 0; v < n; ++v) r[v] += dr[v];
    }
    free(dr); free(rv); free(dv);
    return rc;
}

/* The synchronous iterations of orc_fw_sync with the pairs of an iteration
 * split into `threads` contiguous chunks run by host threads (OpenMP when the
 * oracle is built with it, one after the other otherwise).  Each chunk sums its
 * pairs' allocations into its own delta vector and the vectors are added after
 * the iteration: integer sums, so r_T equals orc_fw_sync's exactly.  Timing
 * baseline only; the pins test it against orc_fw_sync. */
int orc_fw_sync_par(int64_t n, int64_t npairs, const int64_t *pair_off, const int32_t *nodes,
                    const int32_t *hcnt, int k, int T, uint64_t *r, int threads) {
    if (threads < 1) threads = 1;
    const int mx = max_pair_len(npairs, pair_off);
    const size_t stride = (size_t)n + 1;
    uint64_t *dr = (uint64_t *)malloc(sizeof(uint64_t) * stride * (size_t)threads);
    int *crc = (int *)calloc((size_t)threads, sizeof(int));
    if (!dr || !crc) { free(dr); free(crc); return ORC_OVERFLOW; }
    int rc = ORC_OK;
    for (int t = 1; t <= T && rc == ORC_OK; ++t) {
        memset(dr, 0, sizeof(uint64_t) * stride * (size_t)threads);
#pragma omp parallel for num_threads(threads) schedule(static, 1)
        for (int c = 0; c < threads; ++c) {
            uint64_t *d = dr + (size_t)c * stride;
            uint64_t *rv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mx + 1));
            uint64_t *dv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mx + 1));
            const int64_t q0 = npairs * c / threads, q1 = npairs * (c + 1) / threads;
            for (int64_t q = q0; q < q1 && crc[c] == ORC_OK; ++q) {
                const int len = (int)(pair_off[q + 1] - pair_off[q]);
                const int32_t *ids = nodes + pair_off[q];
                for (int i = 0; i < len; ++i) rv[i] = r[ids[i]];
                crc[c] = orc_pbupdate_alg3(len, ids, rv, hcnt[q], k, dv);
                if (crc[c] == ORC_OK)
                    for (int i = 0; i < len; ++i) d[ids[i]] += dv[i];
            }
            free(rv); free(dv);
        }
        for (int c = 0; c < threads; ++c) if (crc[c]) rc = crc[c];
#pragma omp parallel for num_threads(threads) schedule(static)
        for (int64_t v = 0; v < n; ++v) {
            uint64_t x = 0;
            for (int c = 0; c < threads; ++c) x += dr[(size_t)c * stride + (size_t)v];
            r[v] += x;
        }
    }
    free(dr); free(crc);
    return rc;
}

/* Sequential iterations: Alg. 2 as printed updates r in place, pair by    */
/* pair, here in array order.                                               */
int orc_fw_seq(int64_t n, int64_t npairs, const int64_t *pair_off, const int32_t *nodes,
               const int32_t *hcnt, int k, int T, uint64_t *r) {
    (void)n;
    int mx = max_pair_len(npairs, pair_off);
    uint64_t *rv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mx + 1));
    uint64_t *dv = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(mx + 1));
    int rc = ORC_OK;
    for (int t = 1; t <= T && rc == ORC_OK; ++t) {
        for (int64_t q = 0; q < npairs; ++q) {
            int len = (int)(pair_off[q + 1] - pair_off[q]);
            const int32_t *ids = nodes + pair_off[q];
            for (int i = 0; i < len; ++i) rv[i] = r[ids[i]];
            rc = orc_pbupdate_alg3(len, ids, rv, hcnt[q], k, dv);
            if (rc) break;
            for (int i = 0; i < len; ++i) r[ids[i]] += dv[i];
        }
    }
    free(rv); free(dv);
    return rc;
}

/* Synchronous iterations of the continuous rule, FP64, cumulative r. */
int orc_fw_cont(int64_t n, int64_t npairs, const int64_t *pair_off, const int32_t *nodes,
                const int32_t *hcnt, int k, int T, double *r) {
    int mx = max_pair_len(npairs, pair_off);
    double *dr = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *rv = (double *)malloc(sizeof(double) * (size_t)(mx + 1));
    double *dv = (double *)malloc(sizeof(double) * (size_t)(mx + 1));
    int rc = ORC_OK;
    for (int t = 1; t <= T && rc == ORC_OK; ++t) {
        memset(dr, 0, sizeof(double) * (size_t)n);
        for (int64_t q = 0; q < npairs; ++q) {
            int len = (int)(pair_off[q + 1] - pair_off[q]);
            const int32_t *ids = nodes + pair_off[q];
            for (int i = 0; i < len; ++i) rv[i] = r[ids[i]];
            rc = orc_pbupdate_cont(len, ids, rv, hcnt[q], k, dv);
            if (rc) break;
            for (int i = 0; i < len; ++i) dr[ids[i]] += dv[i];
        }
        for (int64_t v = 0; v < n; ++v) r[v] += dr[v];
    }
    free(dr); free(rv); free(dv);
    return rc;
}

/* orc_fw_cont with the per-pair water levels of an iteration computed on
 * host threads (OpenMP when available) into one buffer, then added into the
 * delta vector in pair order by one thread: the same additions in the same
 * order as orc_fw_cont, so r is bit for bit equal (pinned); only faster. */
int orc_fw_cont_par(int64_t n, int64_t npairs, const int64_t *pair_off, const int32_t *nodes,
                    const int32_t *hcnt, int k, int T, double *r, int threads) {
    if (threads < 1) threads = 1;
    const int64_t L = npairs > 0 ? pair_off[npairs] : 0;
    const int mx = max_pair_len(npairs, pair_off);
    double *dr = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double *dall = (double *)malloc(sizeof(double) * (size_t)(L + 1));
    int *crc = (int *)calloc((size_t)threads, sizeof(int));
    if (!dr || !dall || !crc) { free(dr); free(dall); free(crc); return ORC_OVERFLOW; }
    int rc = ORC_OK;
    for (int t = 1; t <= T && rc == ORC_OK; ++t) {
#pragma omp parallel for num_threads(threads) schedule(static, 1)
        for (int c = 0; c < threads; ++c) {
            double *rv = (double *)malloc(sizeof(double) * (size_t)(mx + 1));
            const int64_t q0 = npairs * c / threads, q1 = npairs * (c + 1) / threads;
            for (int64_t q = q0; q < q1 && crc[c] == ORC_OK; ++q) {
                const int len = (int)(pair_off[q + 1] - pair_off[q]);
                const int32_t *ids = nodes + pair_off[q];
                for (int i = 0; i < len; ++i) rv[i] = r[ids[i]];
                crc[c] = orc_pbupdate_cont(len, ids, rv, hcnt[q], k, dall + pair_off[q]);
            }
            free(rv);
        }
        for (int c = 0; c < threads; ++c) if (crc[c]) rc = crc[c];
        if (rc) break;
        memset(dr, 0, sizeof(double) * (size_t)n);
        for (int64_t q = 0; q < npairs; ++q) {
            const int len = (int)(pair_off[q + 1] - pair_off[q]);
            const int32_t *ids = nodes + pair_off[q];
            const double *dv = dall + pair_off[q];
            for (int i = 0; i < len; ++i) dr[ids[i]] += dv[i];
        }
        for (int64_t v = 0; v < n; ++v) r[v] += dr[v];
    }
    free(dr); free(dall); free(crc);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* O4: Alg. 1 over the explicit k-clique list, in place: every clique gives */
/* +1 to its node of smallest (r, id).                                      */
/* ------------------------------------------------------------------------ */
void orc_fw_cliques(int64_t c, const int32_t *cl, int k, int T, uint64_t *r) {
    for (int t = 1; t <= T; ++t)
        for (int64_t q = 0; q < c; ++q) {
            const int32_t *C = cl + q * k;
            int32_t b = C[0];
            for (int i = 1; i < k; ++i)
                if (r[C[i]] < r[b] || (r[C[i]] == r[b] && C[i] < b)) b = C[i];
            r[b]++;
        }
}

/* Alg. 1 over the explicit list in the synchronous reading R1: every clique
 * of iteration t looks at r_{t-1} and hands its unit to its member of least
 * (r, id); the units are summed into r_t after the iteration. */
void orc_fw_cliques_sync(int64_t n, int64_t c, const int32_t *cl, int k, int T, uint64_t *r) {
    uint64_t *d = (uint64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
    for (int t = 1; t <= T; ++t) {
        for (int64_t q = 0; q < c; ++q) {
            const int32_t *C = cl + q * k;
            int32_t best = C[0];
            for (int j = 1; j < k; ++j) {
                const int32_t u = C[j];
                if (r[u] < r[best] || (r[u] == r[best] && u < best)) best = u;
            }
            d[best]++;
        }
        for (int64_t v = 0; v < n; ++v) { r[v] += d[v]; d[v] = 0; }
    }
    free(d);
}

/* ------------------------------------------------------------------------ */
/* CPSample (Sec. 5, Alg. 4): greedy colouring, k-color paths, sampling.    */
/* Readings:                                                                */
/*  S1  The colouring is the linear-time greedy one, vertices taken by      */
/*      decreasing rank of the vertex order (the densest core first), each  */
/*      given the smallest colour no coloured neighbour has.                */
/*  S2  A k-color path is a path v_1 .. v_k with strictly increasing colours */
/*      (a clique's members, sorted by colour, form exactly one such path,  */
/*      so uniform paths give uniform cliques).                              */
/*  S3  A sample is one uniformly drawn path: index R in [0, #paths), from  */
/*      one SplitMix64 word x as R = floor((x >> 11) * #paths / 2^53), then */
/*      the path of rank R in the order (start vertex id, then each next    */
/*      vertex in adjacency order) -- samples are drawn with replacement.    */
/*  S4  The sampled set of k-cliques is a set: repeated cliques count once. */
/* ------------------------------------------------------------------------ */

static int cmp_rank_desc(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return g_key1[x] > g_key1[y] ? -1 : g_key1[x] < g_key1[y];
}

/* S1: colour[v] for every vertex; returns the number of colours. */
int orc_color_greedy(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *rank,
                     int32_t *color) {
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    unsigned char *used = (unsigned char *)calloc((size_t)n + 2, 1);
    for (int64_t v = 0; v < n; ++v) { ord[v] = (int32_t)v; color[v] = -1; }
    g_key1 = rank;
    qsort(ord, (size_t)n, sizeof(int32_t), cmp_rank_desc);
    int ncol = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t v = ord[i];
        for (int64_t e = off[v]; e < off[v + 1]; ++e)
            if (color[adj[e]] >= 0) used[color[adj[e]]] = 1;
        int c = 0;
        while (used[c]) ++c;
        color[v] = c;
        if (c + 1 > ncol) ncol = c + 1;
        for (int64_t e = off[v]; e < off[v + 1]; ++e)
            if (color[adj[e]] >= 0) used[color[adj[e]]] = 0;
    }
    free(ord); free(used);
    return ncol;
}

/* S2: dp[v * k + (i - 1)] = number of increasing-colour paths of i vertices
 * starting at v (i = 1..k).  Returns ORC_OVERFLOW when a count needs more
 * than 64 bits. */
int orc_ccpath_dp(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *color, int k,
                  uint64_t *dp) {
    for (int64_t v = 0; v < n; ++v) dp[v * k] = 1;
    for (int i = 2; i <= k; ++i)
        for (int64_t v = 0; v < n; ++v) {
            unsigned __int128 sum = 0;
            for (int64_t e = off[v]; e < off[v + 1]; ++e)
                if (color[adj[e]] > color[v]) sum += dp[(int64_t)adj[e] * k + (i - 2)];
            if (sum >> 64) return ORC_OVERFLOW;
            dp[v * k + (i - 1)] = (uint64_t)sum;
        }
    return ORC_OK;
}

static uint64_t orc_splitmix64(uint64_t seed, uint64_t index) {
    uint64_t z = seed + (index + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* S3: t samples; sample j draws word j of the SplitMix64 generator seeded
 * with `seed`.  paths[j * k ..] receives the path's vertices, clique[j] = 1
 * when they are pairwise adjacent.  *total receives the number of paths. */
int orc_ccpath_sample(int64_t n, const int64_t *off, const int32_t *adj, const int32_t *color,
                      int k, const uint64_t *dp, int64_t t, uint64_t seed, int32_t *paths,
                      uint8_t *clique, uint64_t *total) {
    unsigned __int128 tot = 0;
    for (int64_t v = 0; v < n; ++v) tot += dp[v * k + (k - 1)];
    if (tot >> 64) return ORC_OVERFLOW;
    *total = (uint64_t)tot;
    for (int64_t j = 0; j < t; ++j) {
        int32_t *P = paths + j * k;
        clique[j] = 0;
        if (tot == 0) { for (int i = 0; i < k; ++i) P[i] = -1; continue; }
        const uint64_t x = orc_splitmix64(seed, (uint64_t)j);
        uint64_t R = (uint64_t)(((unsigned __int128)(x >> 11) * tot) >> 53);
        int64_t v = 0;
        while (R >= dp[v * k + (k - 1)]) { R -= dp[v * k + (k - 1)]; ++v; }
        P[0] = (int32_t)v;
        for (int i = k - 1; i >= 1; --i) {         /* i vertices still to choose */
            for (int64_t e = off[v]; e < off[v + 1]; ++e) {
                const int32_t w = adj[e];
                if (color[w] <= color[v]) continue;
                const uint64_t c = dp[(int64_t)w * k + (i - 1)];
                if (R < c) { v = w; break; }
                R -= c;
            }
            P[k - i] = (int32_t)v;
        }
        int ok = 1;
        for (int a = 0; a < k && ok; ++a)
            for (int b = a + 2; b < k && ok; ++b) {   /* consecutive ones are adjacent */
                int found = 0;
                for (int64_t e = off[P[a]]; e < off[P[a] + 1]; ++e)
                    if (adj[e] == P[b]) { found = 1; break; }
                ok = found;
            }
        clique[j] = (uint8_t)ok;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* O5: extraction (the final sort and prefix step of Alg. 2, R4, R5).      */
/* ------------------------------------------------------------------------ */
static const double *g_key_d;
static int cmp_desc_d(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_key_d[x] != g_key_d[y]) return g_key_d[x] > g_key_d[y] ? -1 : 1;
    return x < y ? -1 : x > y;
}
static const uint64_t *g_key_u;
static int cmp_desc_u(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_key_u[x] != g_key_u[y]) return g_key_u[x] > g_key_u[y] ? -1 : 1;
    return x < y ? -1 : x > y;
}

/* order[i] = i-th node by (r desc, id asc) */
void orc_sort_desc_u64(int64_t n, const uint64_t *r, int32_t *order) {
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    g_key_u = r;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_desc_u);
}
void orc_sort_desc_f64(int64_t n, const double *r, int32_t *order) {
    for (int64_t i = 0; i < n; ++i) order[i] = (int32_t)i;
    g_key_d = r;
    qsort(order, (size_t)n, sizeof(int32_t), cmp_desc_d);
}

/* C_k(V_i) for i = 0..n from the explicit list: a clique lies in V_i iff   */
/* all its nodes are among the first i, i.e. i > max position.  Output as   */
/* 128-bit values split in lo/hi words.                                      */
void orc_prefix_counts_cliques(int64_t n, const int32_t *order, int64_t c, const int32_t *cl,
                               int k, uint64_t *lo, uint64_t *hi) {
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    u128 *acc = (u128 *)calloc((size_t)(n + 1), sizeof(u128));
    for (int64_t i = 0; i < n; ++i) pos[order[i]] = (int32_t)i;
    for (int64_t q = 0; q < c; ++q) {
        int32_t mp = -1;
        for (int i = 0; i < k; ++i) if (pos[cl[q * k + i]] > mp) mp = pos[cl[q * k + i]];
        acc[mp + 1] += 1;
    }
    for (int64_t i = 1; i <= n; ++i) acc[i] += acc[i - 1];
    for (int64_t i = 0; i <= n; ++i) { lo[i] = (uint64_t)acc[i]; hi[i] = (uint64_t)(acc[i] >> 64); }
    free(pos); free(acc);
}

/* C_k(V_i) from the SCT pairs (Lemma 2.5 partition, Lemma 2.6 counts): a   */
/* pair contributes C(#{V_p nodes in V_i}, k - h) once V_h is inside V_i.   */
/* Also F_i = sum of n_C over pairs with V(P) inside V_i (rho'(V_i) = F_i/i, */
/* Theorem 3.6).                                                            */
int orc_prefix_counts_pairs(int64_t n, const int32_t *order, int64_t npairs,
                            const int64_t *pair_off, const int32_t *nodes, const int32_t *hcnt,
                            int k, uint64_t *lo, uint64_t *hi, uint64_t *flo, uint64_t *fhi) {
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    u128 *acc = (u128 *)calloc((size_t)(n + 2), sizeof(u128));
    u128 *facc = (u128 *)calloc((size_t)(n + 2), sizeof(u128));
    for (int64_t i = 0; i < n; ++i) pos[order[i]] = (int32_t)i;
    int mx = max_pair_len(npairs, pair_off);
    int32_t *pp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(mx + 1));
    for (int64_t q = 0; q < npairs; ++q) {
        int len = (int)(pair_off[q + 1] - pair_off[q]);
        const int32_t *ids = nodes + pair_off[q];
        int h = hcnt[q], p = len - h;
        int32_t mh = -1;
        for (int i = 0; i < h; ++i) if (pos[ids[i]] > mh) mh = pos[ids[i]];
        for (int i = 0; i < p; ++i) pp[i] = pos[ids[h + i]];
        /* sort pivot positions */
        for (int a = 1; a < p; ++a) { int32_t t = pp[a]; int b = a - 1;
            while (b >= 0 && pp[b] > t) { pp[b + 1] = pp[b]; --b; } pp[b + 1] = t; }
        /* f(i) = [i > mh] * C(#{j : pp[j] < i}, k - h) */
        int cnt_below = 0;
        while (cnt_below < p && pp[cnt_below] < mh) cnt_below++;
        u128 prev = binom128(cnt_below, k - h);
        acc[mh + 1] += prev;
        for (int j = cnt_below; j < p; ++j) {
            u128 nv = binom128(j + 1, k - h);
            acc[pp[j] + 1] += nv - prev;
            prev = nv;
        }
        int32_t mall = mh;
        for (int j = 0; j < p; ++j) if (pp[j] > mall) mall = pp[j];
        facc[mall + 1] += binom128(p, k - h);
    }
    for (int64_t i = 1; i <= n; ++i) { acc[i] += acc[i - 1]; facc[i] += facc[i - 1]; }
    for (int64_t i = 0; i <= n; ++i) {
        lo[i] = (uint64_t)acc[i]; hi[i] = (uint64_t)(acc[i] >> 64);
        if (flo) { flo[i] = (uint64_t)facc[i]; fhi[i] = (uint64_t)(facc[i] >> 64); }
    }
    free(pos); free(acc); free(facc); free(pp);
    return ORC_OK;
}

/* a/i > b/j for 128-bit a, b and 63-bit i, j, compared exactly by          */
/* cross-multiplication in 192 bits.                                        */
static int frac_cmp(u128 a, uint64_t i, u128 b, uint64_t j) {
    /* a*j vs b*i; each product split into (hi64, lo128) */
    u128 alo = (u128)(uint64_t)a * j, ahi = (u128)(uint64_t)(a >> 64) * j;
    u128 blo = (u128)(uint64_t)b * i, bhi = (u128)(uint64_t)(b >> 64) * i;
    /* value = ahi * 2^64 + alo */
    u128 a_top = ahi + (alo >> 64), b_top = bhi + (blo >> 64);
    uint64_t a_bot = (uint64_t)alo, b_bot = (uint64_t)blo;
    if (a_top != b_top) return a_top > b_top ? 1 : -1;
    if (a_bot != b_bot) return a_bot > b_bot ? 1 : -1;
    return 0;
}

/* i* = largest i in 1..n maximising counts[i] / i (R5). */
int64_t orc_argmax_density(int64_t n, const uint64_t *lo, const uint64_t *hi) {
    int64_t best = 1;
    for (int64_t i = 1; i <= n; ++i) {
        u128 a = ((u128)hi[i] << 64) | lo[i], b = ((u128)hi[best] << 64) | lo[best];
        if (frac_cmp(a, (uint64_t)i, b, (uint64_t)best) >= 0) best = i;
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Brute force over all subsets of a graph with n <= 24 nodes (definition   */
/* of rho_k and of the k-clique densest subgraph, Def. 2.1; rho' of Thm 3.6).*/
/* items: nitems node masks with weights; F[S] = sum of weights of items    */
/* inside S (subset-sum transform).  Returns the best S: maximal density,   */
/* and among the maximisers the largest (the union of all maximisers is     */
/* checked by the caller).                                                  */
/* ------------------------------------------------------------------------ */
int orc_brute_best(int n, int64_t nitems, const uint32_t *masks, const uint64_t *weights,
                   uint32_t *best_mask, uint64_t *best_num, uint64_t *best_den,
                   uint32_t *union_of_maximisers) {
    if (n > 24) return ORC_BAD_GRAPH;
    size_t N = (size_t)1 << n;
    u128 *F = (u128 *)calloc(N, sizeof(u128));
    if (!F) return ORC_OOM;
    for (int64_t q = 0; q < nitems; ++q) F[masks[q]] += weights[q];
    for (int b = 0; b < n; ++b)
        for (size_t S = 0; S < N; ++S)
            if (S & ((size_t)1 << b)) F[S] += F[S ^ ((size_t)1 << b)];
    u128 bn = 0; uint64_t bd = 1; uint32_t bm = 0, uni = 0;
    for (size_t S = 1; S < N; ++S) {
        uint64_t d = (uint64_t)__builtin_popcount((unsigned)S);
        int c = frac_cmp(F[S], d, bn, bd);
        if (c > 0 || (c == 0 && d > bd)) { bn = F[S]; bd = d; bm = (uint32_t)S; }
    }
    for (size_t S = 1; S < N; ++S) {
        uint64_t d = (uint64_t)__builtin_popcount((unsigned)S);
        if (frac_cmp(F[S], d, bn, bd) == 0) uni |= (uint32_t)S;
    }
    *best_mask = bm; *best_num = (uint64_t)bn; *best_den = bd; *union_of_maximisers = uni;
    free(F);
    return ORC_OK;
}
