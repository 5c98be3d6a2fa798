// graph.cu -- steps A1 (simple graph in CSR) and A2 (core numbers, vertex
// order, orientation) of the solver.
//
// A1: the raw edge list becomes the simple undirected graph G(V, E) of Sec. 2:
//     both orientations as 64-bit (u, v) keys, a stable radix sort, duplicate
//     and self-loop removal, row offsets.
// A2: degeneracy (Sec. 2) by round-synchronous peeling in one cooperative
//     kernel: at level c every remaining vertex of remaining degree <= c is
//     removed in one round; vertices whose degree falls to c during a round
//     form the next round's frontier; when none is left, c rises to the
//     smallest remaining degree.  The build order is (round, id) or
//     (core, id); the out-CSR keeps u -> w iff w is later than u.
#include <algorithm>

#include "graph.cuh"

namespace kdss {

namespace {

constexpr uint64_t SENT = ~0ull;

__global__ void k_edge_keys(const int32_t *src, const int32_t *dst, int64_t m, int64_t n,
                            uint64_t *keys, int *err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t u = src[e], v = dst[e];
        uint64_t a = SENT, b = SENT;
        if (u < 0 || v < 0 || u >= n || v >= n) {
            atomicOr(err, DERR_BAD_ID);
        } else if (u != v) {
            a = ((uint64_t)u << 32) | (uint64_t)v;
            b = ((uint64_t)v << 32) | (uint64_t)u;
        }
        keys[2 * e] = a;
        keys[2 * e + 1] = b;
    }
}

__global__ void k_unique_flags(const uint64_t *keys, int64_t nk, int64_t *flags) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nk;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        flags[i] = (k != SENT && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
}

__global__ void k_compact_keys(const uint64_t *keys, int64_t nk, const int64_t *flags,
                               const int64_t *pos, uint64_t *ukeys, int32_t *adj) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nk;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (flags[i]) {
            uint64_t k = keys[i];
            ukeys[pos[i]] = k;
            if (adj) adj[pos[i]] = (int32_t)(k & 0xffffffffu);
        }
    }
}

__global__ void k_degrees(const int64_t *off, int64_t n, int32_t *deg, int32_t *rnd) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        deg[v] = (int32_t)(off[v + 1] - off[v]);
        rnd[v] = -1;
    }
}

struct PeelCtl {
    GridBarrier bar;
    int err;
    int acnt[2];              // appends of the rounds of each parity (never reset)
    unsigned int minval;
    int rounds;
    int degeneracy;
    int pub_round, pub_start, pub_end;   // state after such a run
};

constexpr int PEEL_THREADS = 1024;
// Frontiers of at most this many vertices are removed by block 0 alone, one
// round after another with block barriers, while the other blocks wait at
// the next grid barrier: most rounds of a power-law graph are a few vertices
// at the end of a level, and there a round costs its chain of dependent
// loads and atomics, not its work.
constexpr int PEEL_SMALL = 128;

// Remove the frontier cur[0, cnt): warps [warp0, warp0 + nwarps) take its
// vertices; every neighbour loses one degree, and one that falls from
// level + 1 to level joins the next round: it is written to the peel order
// at position atomicAdd(counter, 1) + pos_off.  Neighbours already removed or
// queued are decremented too: their degree is at most the level they were
// taken at, which is at most `level`, so it never again equals level + 1, and
// nothing reads it afterwards; skipping the check saves a dependent load of
// rnd per neighbour.
__device__ __forceinline__ void peel_remove(int cnt, int64_t warp0, int64_t nwarps,
                                            const longlong2 *cur, longlong2 *order,
                                            const int64_t *__restrict__ off,
                                            const int32_t *__restrict__ adj, int32_t *deg,
                                            int32_t *rnd, int32_t *core, int *counter,
                                            int64_t pos_off, int64_t n, int level, int round) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = warp0; i < cnt; i += nwarps) {
        const longlong2 er = __ldcg(cur + i);
        const int64_t e0 = er.x, e1 = er.y;
        // four neighbours per lane at a time: their loads and atomics are
        // independent and overlap (hubs have thousands of neighbours)
        for (int64_t e = e0 + lane; e < e1; e += 128) {
            int32_t w[4];
            int old[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t ee = e + 32 * u;
                w[u] = ee < e1 ? adj[ee] : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) old[u] = w[u] >= 0 ? atomicSub(deg + w[u], 1) : 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (w[u] >= 0 && old[u] == level + 1) {
                    rnd[w[u]] = round + 1;
                    core[w[u]] = level;
                    const int64_t idx = (int64_t)atomicAdd(counter, 1) + pos_off;
                    if (idx >= 0 && idx < n) order[idx] = make_longlong2(off[w[u]], off[w[u] + 1]);
                }
            }
        }
    }
}

// A run of small rounds in block 0 alone, while the other blocks wait at a
// grid barrier.  The frontier lives in shared memory as the edge ranges of its
// vertices; a vertex that joins the next round takes a slot from a shared
// counter, is written to the peel order after the current frontier (where the
// grid reads it if the run stops) and, while the next frontier has room, to
// the other shared buffer with its edge range.  A round is then a chain of
// three global accesses (the neighbour list, the atomic decrement, the edge
// range of a joining vertex) and two block barriers.  On return order[s, e)
// is the next frontier (empty, or larger than PEEL_SMALL) and `round` its
// round.  Every thread of block 0 calls this.
__device__ __forceinline__ void peel_local_run(int64_t &s, int64_t &e, int &round, int level,
                                               int64_t n, const int64_t *__restrict__ off,
                                               const int32_t *__restrict__ adj, int32_t *deg,
                                               int32_t *rnd, int32_t *core, longlong2 *order,
                                               PeelCtl *ctl) {
    __shared__ long long le0[2][PEEL_SMALL], le1[2][PEEL_SMALL];
    __shared__ int lcnt[2];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < (int)(e - s); i += blockDim.x) {
        const longlong2 er = __ldcg(order + s + i);
        le0[0][i] = er.x;
        le1[0][i] = er.y;
    }
    if (threadIdx.x == 0) {
        lcnt[0] = 0;
        lcnt[1] = 0;
    }
    __syncthreads();
    int cur = 0;
    while (true) {
        const int cnt = (int)(e - s), nx = cur ^ 1;
        for (int i = wib; i < cnt; i += nw) {
            const int64_t e0 = le0[cur][i], e1 = le1[cur][i];
            for (int64_t x = e0 + lane; x < e1; x += 128) {
                int32_t w[4];
                int old[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) w[u] = x + 32 * u < e1 ? adj[x + 32 * u] : -1;
#pragma unroll
                for (int u = 0; u < 4; ++u) old[u] = w[u] >= 0 ? atomicSub(deg + w[u], 1) : 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (w[u] >= 0 && old[u] == level + 1) {
                        rnd[w[u]] = round + 1;
                        core[w[u]] = level;
                        const int slot = atomicAdd(&lcnt[nx], 1);
                        const long long a0 = off[w[u]], a1 = off[w[u] + 1];
                        if (e + slot < n) order[e + slot] = make_longlong2(a0, a1);
                        if (slot < PEEL_SMALL) {
                            le0[nx][slot] = a0;
                            le1[nx][slot] = a1;
                        }
                    }
                }
            }
        }
        if (threadIdx.x == 0) {
            if (level > ctl->degeneracy) ctl->degeneracy = level;
            ctl->rounds = round + 1;
        }
        __syncthreads();
        const int next = lcnt[nx];
        if (threadIdx.x == 0) lcnt[cur] = 0;   // read by everyone before the barrier above
        __syncthreads();
        ++round;
        s = e;
        e = e + next < n ? e + next : n;   // (appends beyond n are dropped; caught by the caller)
        cur = nx;
        if (next == 0 || next > PEEL_SMALL) break;   // uniform in the block
    }
}

// The frontiers are consecutive ranges of one array, the peel order, which
// holds each queued vertex as its edge range (off[v], off[v + 1]): a round
// starts from the ranges without a dependent load of off.  Round r
// removes order[S_r, S_{r+1}).  Round r appends through acnt[(r + 1) & 1] and
// round r + 1 reads that counter to find its end, so no round's appends touch
// the counter the same round reads (a late block may still be reading it
// while others append), and no counter is ever reset.  Each block keeps the
// value of each counter it last read; a counter changes only between two of
// its reads, so the differences give the rounds' sizes.  A run of rounds in
// block 0 appends through a shared-memory counter and leaves acnt untouched.
__global__ void __launch_bounds__(PEEL_THREADS, 1)
k_peel(int64_t n, const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
       int32_t *deg, int32_t *rnd, int32_t *core, longlong2 *order, PeelCtl *ctl,
       uint64_t timeout_ns, unsigned int phantom) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    // phantom > 0 (failure-injection test only): the barriers wait for blocks
    // that do not exist, so the first wait expires in every block
    const unsigned int nb = gridDim.x + phantom;
    unsigned int epoch = 0;      // grid barriers passed (the host clears the counter)
    int level = 0, round = 0;
    int64_t S = 0, E = 0;        // this round's frontier: order[S, E)
    int last0 = 0, last1 = 0;    // acnt[0], acnt[1] as this block last read them
    bool have_end = false;       // E already known (after a run in block 0)
    volatile int *vacnt = ctl->acnt;
    while (true) {
        const int pr = round & 1;
        if (!have_end) {
            const int a = vacnt[pr];
            E = S + (a - (pr ? last1 : last0));
            if (pr) last1 = a; else last0 = a;
        }
        have_end = false;
        if (E > n || E < S) { if (tid == 0) atomicOr(&ctl->err, DERR_CAPACITY); return; }  // uniform
        if (E == S) {
            if (S >= n) break;
            // smallest remaining degree
            unsigned int mn = 0xffffffffu;
            for (int64_t v = tid; v < n; v += nth)
                if (__ldcg(rnd + v) < 0) {
                    unsigned int d = (unsigned int)__ldcg(deg + v);
                    mn = d < mn ? d : mn;
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                unsigned int t = __shfl_xor_sync(0xffffffffu, mn, o);
                mn = t < mn ? t : mn;
            }
            if ((threadIdx.x & 31) == 0 && mn != 0xffffffffu) atomicMin(&ctl->minval, mn);
            if (!grid_sync_count(&ctl->bar.count, ++epoch * nb, &ctl->err, timeout_ns)) return;
            unsigned int mv = *(volatile unsigned int *)&ctl->minval;
            if (mv == 0xffffffffu) {  // nothing alive: inconsistent counters
                if (tid == 0) atomicOr(&ctl->err, DERR_LOGIC);
                return;
            }
            if ((int)mv > level) level = (int)mv;
            // the new level's first frontier, through acnt[pr] (everyone read
            // it before the barrier above)
            const int64_t base = S - (pr ? last1 : last0);
            for (int64_t v = tid; v < n; v += nth)
                if (__ldcg(rnd + v) < 0 && __ldcg(deg + v) <= level) {
                    const int64_t idx = (int64_t)atomicAdd(&ctl->acnt[pr], 1) + base;
                    if (idx >= 0 && idx < n) order[idx] = make_longlong2(off[v], off[v + 1]);
                    rnd[v] = round;
                    core[v] = level;
                }
            if (!grid_sync_count(&ctl->bar.count, ++epoch * nb, &ctl->err, timeout_ns)) return;
            // minval is next read after at least one more barrier
            if (tid == 0) ctl->minval = 0xffffffffu;
            const int a = vacnt[pr];
            E = S + (a - (pr ? last1 : last0));
            if (pr) last1 = a; else last0 = a;
            if (E > n || E <= S) { if (tid == 0) atomicOr(&ctl->err, DERR_LOGIC); return; }
        }
        if (E - S <= PEEL_SMALL) {
            if (blockIdx.x == 0) {
                // consecutive small rounds in this block alone
                int64_t s = S, e = E;
                peel_local_run(s, e, round, level, n, off, adj, deg, rnd, core, order, ctl);
                if (threadIdx.x == 0) {
                    ctl->pub_round = round;
                    ctl->pub_start = (int)s;
                    ctl->pub_end = (int)e;
                }
            }
            if (!grid_sync_count(&ctl->bar.count, ++epoch * nb, &ctl->err, timeout_ns)) return;
            round = *(volatile int *)&ctl->pub_round;
            S = *(volatile int *)&ctl->pub_start;
            E = *(volatile int *)&ctl->pub_end;
            have_end = true;
            continue;
        }
        // a large frontier: every block; appends through acnt[round + 1 & 1]
        const int64_t pos_off = E - (pr ? last0 : last1);
        peel_remove((int)(E - S), tid >> 5, nth >> 5, order + S, order, off, adj, deg, rnd, core,
                    &ctl->acnt[pr ^ 1], pos_off, n, level, round);
        if (tid == 0) {
            if (level > ctl->degeneracy) ctl->degeneracy = level;
            ctl->rounds = round + 1;
        }
        if (!grid_sync_count(&ctl->bar.count, ++epoch * nb, &ctl->err, timeout_ns)) return;
        S = E;
        ++round;
    }
}

__global__ void k_order_keys(int64_t n, const int32_t *key, uint64_t *keys) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        keys[v] = ((uint64_t)(uint32_t)key[v] << 32) | (uint64_t)v;
}

__global__ void k_order_ranks(int64_t n, const uint64_t *keys, int32_t *vert, int32_t *rank) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = (int32_t)(keys[i] & 0xffffffffu);
        vert[i] = v;
        rank[v] = (int32_t)i;
    }
}

// One flag per CSR entry: keep (v, w) iff rank[v] < rank[w].
__global__ void k_orient_flags(int64_t n, const int64_t *off, const int32_t *adj,
                               const int32_t *rank, int64_t *flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        int32_t rv = rank[v];
        for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32)
            flags[e] = rank[adj[e]] > rv ? 1 : 0;
    }
}

__global__ void k_orient_keys(int64_t n, const int64_t *off, const int32_t *adj,
                              const int32_t *rank, const int64_t *flags, const int64_t *pos,
                              uint64_t *keys) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < n; v += nwarps) {
        uint64_t rv = (uint64_t)(uint32_t)rank[v];
        for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32)
            if (flags[e]) keys[pos[e]] = (rv << 32) | (uint64_t)(uint32_t)rank[adj[e]];
    }
}

__global__ void k_low32(const uint64_t *keys, int64_t nk, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nk;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)(keys[i] & 0xffffffffu);
}

__global__ void k_max_rowlen(const int64_t *off, int64_t n, int *out) {
    int m = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int d = (int)(off[v + 1] - off[v]);
        m = d > m ? d : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

}  // namespace

void build_graph(const Ctx &c, const kdss_graph_desc &g, int order, GraphDev &out) {
    const int64_t n = g.n, m = g.m;
    out.n = n;
    const int B = 256;
    DBuf<int> err(c, 1);
    zero(c, err.p, sizeof(int));

    // ---- A1: symmetric, deduplicated CSR -------------------------------
    DBuf<int32_t> hsrc, hdst;
    const int32_t *src = g.src, *dst = g.dst;
    if (!g.on_device && m > 0) {
        hsrc = DBuf<int32_t>(c, (size_t)m);
        hdst = DBuf<int32_t>(c, (size_t)m);
        to_device(c, hsrc.p, g.src, (size_t)m);
        to_device(c, hdst.p, g.dst, (size_t)m);
        src = hsrc.p;
        dst = hdst.p;
    }
    const int64_t nk = 2 * m;
    DBuf<uint64_t> keys(c, (size_t)std::max<int64_t>(nk, 1));
    if (m > 0) {
        k_edge_keys<<<grid_for(c, m, B), B, 0, c.stream>>>(src, dst, m, n, keys.p, err.p);
        KDSS_LAUNCH_CHECK();
    }
    hsrc.reset();
    hdst.reset();
    const int b = bit_length((uint64_t)n) + 1;  // sentinel bits sort last
    radix_sort_u64(c, keys.p, nullptr, nk, {{0, b}, {32, 32 + b}});
    DBuf<int64_t> flags(c, (size_t)std::max<int64_t>(nk, 1)), pos(c, (size_t)std::max<int64_t>(nk, 1));
    int64_t nadj = 0;
    if (nk > 0) {
        k_unique_flags<<<grid_for(c, nk, B), B, 0, c.stream>>>(keys.p, nk, flags.p);
        KDSS_LAUNCH_CHECK();
        nadj = exclusive_scan_i64(c, flags.p, pos.p, nk);
    }
    int herr = 0;
    to_host(c, &herr, err.p, 1);
    if (herr & DERR_BAD_ID) fail(KDSS_ERR_BAD_GRAPH, "an edge endpoint is outside [0, n)");
    out.nadj = nadj;
    out.off = DBuf<int64_t>(c, (size_t)(n + 1));
    out.adj = DBuf<int32_t>(c, (size_t)std::max<int64_t>(nadj, 1));
    DBuf<uint64_t> ukeys(c, (size_t)std::max<int64_t>(nadj, 1));
    if (nk > 0) {
        k_compact_keys<<<grid_for(c, nk, B), B, 0, c.stream>>>(keys.p, nk, flags.p, pos.p,
                                                               ukeys.p, out.adj.p);
        KDSS_LAUNCH_CHECK();
    }
    keys.reset();
    row_offsets_from_sorted(c, ukeys.p, nadj, n, out.off.p);
    ukeys.reset();

    // ---- A2: peeling (cooperative kernel, bounded barriers) -------------
    out.core = DBuf<int32_t>(c, (size_t)std::max<int64_t>(n, 1));
    out.rnd = DBuf<int32_t>(c, (size_t)std::max<int64_t>(n, 1));
    if (n > 0) {
        DBuf<int32_t> deg(c, (size_t)n);
        DBuf<longlong2> order(c, (size_t)n);
        DBuf<PeelCtl> ctl(c, 1);
        zero(c, ctl.p, sizeof(PeelCtl));
        unsigned int ff = 0xffffffffu;
        KDSS_CUDA(cudaMemcpyAsync(&ctl.p->minval, &ff, sizeof ff, cudaMemcpyHostToDevice, c.stream));
        k_degrees<<<grid_for(c, n, B), B, 0, c.stream>>>(out.off.p, n, deg.p, out.rnd.p);
        KDSS_LAUNCH_CHECK();
        // One block per SM at most: every round ends in a grid barrier whose
        // cost grows with the number of arriving blocks.
        int per_sm = 0;
        KDSS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel, PEEL_THREADS, 0));
        if (per_sm < 1) fail(KDSS_ERR_CUDA, "peeling kernel cannot be resident");
        int grid = (int)std::min<int64_t>((int64_t)c.num_sms,
                                          std::max<int64_t>(1, ceil_div(n, PEEL_THREADS)));
        uint64_t timeout_ns = 20ull * 1000 * 1000 * 1000;  // 20 s per barrier wait
        unsigned int phantom = 0;
        if (c.flags & KDSS_FLAG_TEST_BARRIER_TIMEOUT) {  // failure injection: 1 ms waits that expire
            timeout_ns = 1000ull * 1000;
            phantom = 1;
        }
        int64_t nn = n;
        const int64_t *offp = out.off.p;
        const int32_t *adjp = out.adj.p;
        int32_t *degp = deg.p, *rndp = out.rnd.p, *corep = out.core.p;
        longlong2 *orderp = order.p;
        PeelCtl *ctlp = ctl.p;
        void *args[] = {&nn, &offp, &adjp, &degp, &rndp, &corep, &orderp, &ctlp, &timeout_ns,
                        &phantom};
        KDSS_CUDA(cudaLaunchCooperativeKernel((const void *)k_peel, dim3(grid), dim3(PEEL_THREADS),
                                              args, 0, c.stream));
        KDSS_LAUNCH_CHECK();
        PeelCtl h;
        to_host(c, &h, ctl.p, 1);
        if (h.err & DERR_TIMEOUT) fail(KDSS_ERR_TIMEOUT, "peeling: a grid barrier wait expired");
        if (h.err) fail(KDSS_ERR_CUDA, "peeling: inconsistent device state");
        out.degeneracy = h.degeneracy;
        out.peel_rounds = h.rounds;
    }

    // ---- A2: vertex order and rank-space out-CSR ------------------------
    out.rank = DBuf<int32_t>(c, (size_t)std::max<int64_t>(n, 1));
    out.vert = DBuf<int32_t>(c, (size_t)std::max<int64_t>(n, 1));
    if (n > 0) {
        DBuf<uint64_t> okeys(c, (size_t)n);
        const int32_t *key = order == KDSS_ORDER_CORE ? out.core.p : out.rnd.p;
        k_order_keys<<<grid_for(c, n, B), B, 0, c.stream>>>(n, key, okeys.p);
        KDSS_LAUNCH_CHECK();
        // the keys are written in id order and the sort is stable, so the
        // high word alone (round or core) gives the (key, id) order
        int kb = bit_length((uint64_t)std::max<int64_t>(out.peel_rounds, out.degeneracy) + 1);
        radix_sort_u64(c, okeys.p, nullptr, n, {{32, 32 + kb}});
        k_order_ranks<<<grid_for(c, n, B), B, 0, c.stream>>>(n, okeys.p, out.vert.p, out.rank.p);
        KDSS_LAUNCH_CHECK();
    }
    int64_t m1 = 0;
    DBuf<uint64_t> okeys;
    if (nadj > 0) {
        k_orient_flags<<<grid_for(c, n * 32, B), B, 0, c.stream>>>(n, out.off.p, out.adj.p,
                                                                  out.rank.p, flags.p);
        KDSS_LAUNCH_CHECK();
        m1 = exclusive_scan_i64(c, flags.p, pos.p, nadj);
        okeys = DBuf<uint64_t>(c, (size_t)std::max<int64_t>(m1, 1));
        k_orient_keys<<<grid_for(c, n * 32, B), B, 0, c.stream>>>(n, out.off.p, out.adj.p,
                                                                 out.rank.p, flags.p, pos.p,
                                                                 okeys.p);
        KDSS_LAUNCH_CHECK();
        radix_sort_u64(c, okeys.p, nullptr, m1, {{0, b}, {32, 32 + b}});
    }
    flags.reset();
    pos.reset();
    out.out_off = DBuf<int64_t>(c, (size_t)(n + 1));
    out.out_adj = DBuf<int32_t>(c, (size_t)std::max<int64_t>(m1, 1));
    row_offsets_from_sorted(c, okeys.p, m1, n, out.out_off.p);
    if (m1 > 0) {
        k_low32<<<grid_for(c, m1, B), B, 0, c.stream>>>(okeys.p, m1, out.out_adj.p);
        KDSS_LAUNCH_CHECK();
    }
    DBuf<int> mx(c, 1);
    zero(c, mx.p, sizeof(int));
    if (n > 0) {
        k_max_rowlen<<<grid_for(c, n, B), B, 0, c.stream>>>(out.out_off.p, n, mx.p);
        KDSS_LAUNCH_CHECK();
    }
    to_host(c, &out.max_out, mx.p, 1);
}

}  // namespace kdss
