// batch.cu -- kdss_solve_batch: many (graph, k, T) queries in one pass.
//
// Queries that share (k, T) form a group whose graphs are joined into one
// disjoint union (node ids shifted by the running node count).  Peeling is
// local to connected components: a component loses the same vertices in the
// same order of rounds inside the union as alone, only at later global round
// numbers, and the shifted ids keep their order; so the (round, id) order of
// the union restricted to a component is the component's own order, and the
// union's SCT is the union of the per-graph SCTs with shifted ids.  One CSR
// build, one peeling and one SCT build then serve the whole group.
//
// All groups iterate together on one state vector: an iteration launches
// every active group's PBUpdate kernels on its slice of r (a pointer offset)
// and steps each slice; the iteration is captured once as a CUDA graph and
// replayed.  Groups with a smaller T leave the graph after T iterations.
//
// Extraction is segmented by query: a stable radix sort by (r desc) and then
// by query index gives every query's node order; the prefix-count increments
// of the pairs land in one histogram whose query segments are n_q + 1 long;
// after one scan, one block per query finds its best prefix exactly.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>

#include "handles.cuh"

namespace kdss {

void extract_prefix(const Ctx &c, const SctDev &s, const StateDev &st, kdss_result *out);

// What the batch autotuner tried (chunk, lanes per long pair, ms of one
// iteration) and what it chose; kept per host thread for kdss_batch_tuning.
struct BatchTuning {
    bool done = false;
    int chunk = 0, tpp = 0;
    struct Tried { int chunk, tpp; float ms; };
    std::vector<Tried> tried;
};
namespace {
thread_local BatchTuning g_last_tuning;
}
void set_last_batch_tuning(const BatchTuning &t) { g_last_tuning = t; }
const BatchTuning &last_batch_tuning() { return g_last_tuning; }

namespace {

constexpr unsigned FULL = 0xffffffffu;

// one query of a union: where its edges are and where its nodes go
struct Member {
    const int32_t *src, *dst;
    int64_t m, n, base, eoff;  // edges, nodes, node base, first edge in the union
};

// shift every query's edges into the union; ids outside [0, n_q) become a
// self-loop of the query's base node (dropped by the CSR build) and flag it
__global__ void k_union_edges(const Member *mem, int nmem, int64_t m_all, int32_t *usrc,
                              int32_t *udst, int *bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m_all;
         e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nmem - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (mem[mid].eoff <= e) lo = mid; else hi = mid - 1;
        }
        const Member &q = mem[lo];
        const int64_t j = e - q.eoff;
        const int64_t u = q.src[j], v = q.dst[j];
        if (u < 0 || v < 0 || u >= q.n || v >= q.n) {
            bad[lo] = 1;
            usrc[e] = (int32_t)q.base;
            udst[e] = (int32_t)q.base;
        } else {
            usrc[e] = (int32_t)(q.base + u);
            udst[e] = (int32_t)(q.base + v);
        }
    }
}

// per node: index of its query inside the group
__global__ void k_node_query(const int64_t *qbase, int nqg, int64_t n, int32_t *qof) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = nqg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (qbase[mid] <= v) lo = mid; else hi = mid - 1;
        }
        qof[v] = lo;
    }
}

// key of r as an order-preserving unsigned value
__device__ __forceinline__ uint64_t rkey(const void *r, int prec, int64_t v) {
    if (prec == KDSS_FP32K) {
        const float x = static_cast<const float *>(r)[v];
        return x > 0.f ? (uint64_t)(uint32_t)__float_as_int(x) : 0ull;
    }
    return static_cast<const uint64_t *>(r)[v];  // uint64, or the bits of a double >= 0
}

// one block per query: max key over its node range
__global__ void k_query_max(const void *r, int prec, const int64_t *qbase, const int64_t *qn,
                            unsigned long long *qmax) {
    const int q = blockIdx.x;
    unsigned long long m = 0;
    for (int64_t i = threadIdx.x; i < qn[q]; i += blockDim.x) {
        const unsigned long long k = rkey(r, prec, qbase[q] + i);
        m = k > m ? k : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(FULL, m, o);
        m = t > m ? t : m;
    }
    __shared__ unsigned long long sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = sm[w] > m ? sm[w] : m;
        m = sm[0] > m ? sm[0] : m;
        qmax[q] = m;
    }
}

__global__ void k_desc_keys(const void *r, int prec, int64_t n, const int32_t *qof,
                            const unsigned long long *qmax, uint64_t *keys, int32_t *vals) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        keys[v] = qmax[qof[v]] - rkey(r, prec, v);
        vals[v] = (int32_t)v;
    }
}

__global__ void k_query_keys(int64_t n, const int32_t *order, const int32_t *qof, uint64_t *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        keys[i] = (uint64_t)qof[order[i]];
}

// histogram position of each node: segment of its query (n_q + 1 slots,
// starting at qbase[q] + q) plus its rank inside the query
__global__ void k_hist_pos(int64_t n, const int32_t *order, const int32_t *qof,
                           const int64_t *qbase, int32_t *pos) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = order[i];
        const int q = qof[v];
        pos[v] = (int32_t)(qbase[q] + q + (i - qbase[q]));
    }
}

__device__ __forceinline__ int frac_cmp(unsigned long long a, unsigned long long i,
                                        unsigned long long b, unsigned long long j) {
    const unsigned long long ahi = __umul64hi(a, j), alo = a * j;
    const unsigned long long bhi = __umul64hi(b, i), blo = b * i;
    if (ahi != bhi) return ahi > bhi ? 1 : -1;
    if (alo != blo) return alo > blo ? 1 : -1;
    return 0;
}
__device__ __forceinline__ void better(unsigned long long &a, long long &i, unsigned long long b,
                                       long long j) {
    if (j <= 0) return;
    if (i <= 0) { a = b; i = j; return; }
    const int c = frac_cmp(b, (unsigned long long)j, a, (unsigned long long)i);
    if (c > 0 || (c == 0 && j > i)) { a = b; i = j; }
}

// one block per query: best prefix of C_k (largest i on ties) and of F
__global__ void k_query_best(const unsigned long long *hist, const unsigned long long *fhist,
                             const int64_t *qbase, const int64_t *qn, unsigned long long *best,
                             long long *bi, unsigned long long *fbest, long long *fi) {
    const int q = blockIdx.x;
    const int64_t hb = qbase[q] + q;
    const unsigned long long h0 = hb > 0 ? hist[hb - 1] : 0ull, f0 = hb > 0 ? fhist[hb - 1] : 0ull;
    unsigned long long a = 0, fa = 0;
    long long i = 0, fi_ = 0;
    for (int64_t j = 1 + threadIdx.x; j <= qn[q]; j += blockDim.x) {
        better(a, i, hist[hb + j] - h0, j);
        better(fa, fi_, fhist[hb + j] - f0, j);
    }
    for (int o = 16; o > 0; o >>= 1) {
        better(a, i, __shfl_xor_sync(FULL, a, o), __shfl_xor_sync(FULL, i, o));
        better(fa, fi_, __shfl_xor_sync(FULL, fa, o), __shfl_xor_sync(FULL, fi_, o));
    }
    __shared__ unsigned long long sa[32], sfa[32];
    __shared__ long long si[32], sfi[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sa[w] = a; si[w] = i; sfa[w] = fa; sfi[w] = fi_; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int x = 0; x < (int)(blockDim.x >> 5); ++x) {
            better(a, i, sa[x], si[x]);
            better(fa, fi_, sfa[x], sfi[x]);
        }
        best[q] = a; bi[q] = i; fbest[q] = fa; fi[q] = fi_;
    }
}

}  // namespace

// defined in extract.cu (same semantics as its use there)
void launch_prefix_events_all(const Ctx &c, const SctDev &s, const int32_t *pos,
                              unsigned long long *hist, unsigned long long *fhist);

namespace {

struct Group {
    int k = 0, T = 0;
    std::vector<int> members;        // query indices
    std::vector<int64_t> qbase, qn;  // node base and n of each member inside the union
    int64_t n = 0;                   // nodes of the union
    int64_t node_off = 0;            // slice of the shared state
    bool skip = false;               // every member failed before the iterations
    SctDev s;
};

void extract_group(const Ctx &c, Group &g, StateDev &st, kdss_result *out) {
    const int nqg = (int)g.members.size();
    const int64_t n = g.n;
    if (n == 0) {
        for (int i : g.members) {
            memset(&out[i], 0, sizeof out[i]);
            out[i].T = g.T;
            out[i].t_used = st.t;
        }
        return;
    }
    const int prec = st.precision;
    const void *r = prec == KDSS_FP32K ? (const void *)(st.r32.p + g.node_off)
                                       : (const void *)(st.r.p + g.node_off);
    const int B = 256;
    DBuf<int64_t> qb(c, nqg), qn(c, nqg);
    to_device(c, qb.p, g.qbase.data(), nqg);
    to_device(c, qn.p, g.qn.data(), nqg);
    DBuf<int32_t> qof(c, n);
    k_node_query<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(qb.p, nqg, n, qof.p);
    KDSS_LAUNCH_CHECK();
    DBuf<unsigned long long> qmax(c, nqg);
    k_query_max<<<nqg, 256, 0, c.stream>>>(r, prec, qb.p, qn.p, qmax.p);
    KDSS_LAUNCH_CHECK();
    std::vector<unsigned long long> hmax(nqg);
    to_host(c, hmax.data(), qmax.p, nqg);
    unsigned long long top = 0;
    for (auto v : hmax) top = std::max(top, v);
    DBuf<uint64_t> keys(c, n);
    DBuf<int32_t> order(c, n);
    k_desc_keys<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(r, prec, n, qof.p, qmax.p, keys.p, order.p);
    KDSS_LAUNCH_CHECK();
    radix_sort_u64(c, keys.p, order.p, n, {{0, bit_length(top)}});
    k_query_keys<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, order.p, qof.p, keys.p);
    KDSS_LAUNCH_CHECK();
    radix_sort_u64(c, keys.p, order.p, n, {{0, bit_length((uint64_t)nqg)}});
    DBuf<int32_t> pos(c, n);
    k_hist_pos<<<grid_for(c, n, B, 4), B, 0, c.stream>>>(n, order.p, qof.p, qb.p, pos.p);
    KDSS_LAUNCH_CHECK();
    const int64_t hn = n + nqg + 1;
    DBuf<unsigned long long> hist(c, hn), fhist(c, hn);
    zero(c, hist.p, hn * 8);
    zero(c, fhist.p, hn * 8);
    launch_prefix_events_all(c, g.s, pos.p, hist.p, fhist.p);
    inclusive_scan_u64_async(c, (const uint64_t *)hist.p, (uint64_t *)hist.p, hn);
    inclusive_scan_u64_async(c, (const uint64_t *)fhist.p, (uint64_t *)fhist.p, hn);
    DBuf<unsigned long long> best(c, nqg), fbest(c, nqg);
    DBuf<long long> bi(c, nqg), fi(c, nqg);
    k_query_best<<<nqg, 256, 0, c.stream>>>(hist.p, fhist.p, qb.p, qn.p, best.p, bi.p, fbest.p, fi.p);
    KDSS_LAUNCH_CHECK();
    std::vector<unsigned long long> hb(nqg), hfb(nqg);
    std::vector<long long> hbi(nqg), hfi(nqg);
    to_host(c, hb.data(), best.p, nqg);
    to_host(c, hbi.data(), bi.p, nqg);
    to_host(c, hfb.data(), fbest.p, nqg);
    to_host(c, hfi.data(), fi.p, nqg);
    const int t = st.t;
    for (int j = 0; j < nqg; ++j) {
        kdss_result &o = out[g.members[j]];
        memset(&o, 0, sizeof o);
        o.T = g.T;
        o.t_used = t;
        double um;
        if (prec == KDSS_FP32K) {
            const uint32_t b32 = (uint32_t)hmax[j];
            float f;
            memcpy(&f, &b32, 4);
            um = f;
        } else if (prec == KDSS_FP64) {
            double d;
            memcpy(&d, &hmax[j], 8);
            um = t > 0 ? d / t : 0.0;
        } else {
            um = t > 0 ? (double)hmax[j] / t : 0.0;
        }
        o.istar = g.qn[j] > 0 ? hbi[j] : 0;
        o.count_lo = g.qn[j] > 0 ? hb[j] : 0;
        o.density = o.istar > 0 ? (double)o.count_lo / (double)o.istar : 0.0;
        o.upper_bound = um;
        o.rho_prime = hfi[j] > 0 ? (double)hfb[j] / (double)hfi[j] : 0.0;
        o.gap = um > 0 ? 1.0 - o.rho_prime / um : 0.0;
        o.status = KDSS_OK;
        if (o.istar > 0) {
            o.ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)o.istar);
            if (!o.ids) fail(KDSS_ERR_OOM, "host allocation of the result ids");
            to_host(c, o.ids, order.p + g.qbase[j], (size_t)o.istar);
            for (int64_t x = 0; x < o.istar; ++x) o.ids[x] -= (int32_t)g.qbase[j];
            std::sort(o.ids, o.ids + o.istar);
        }
    }
}

}  // namespace

void solve_batch(const kdss_query *q, int nq, kdss_result *out, const kdss_opts *opts,
                 std::vector<kdss_status> &status, std::vector<std::string> &msgs) {
    Ctx c = make_ctx(opts);
    const int prec = opts ? opts->precision : KDSS_INT64;
    const int order = opts ? opts->order : KDSS_ORDER_PEEL;
    if (prec != KDSS_INT64 && prec != KDSS_FP64 && prec != KDSS_FP32K)
        fail(KDSS_ERR_INVALID_ARG, "unknown precision");
    status.assign(nq, KDSS_OK);
    msgs.assign(nq, "");
    for (int i = 0; i < nq; ++i) memset(&out[i], 0, sizeof out[i]);
    // groups by (k, T)
    std::map<std::pair<int, int>, Group> groups;
    for (int i = 0; i < nq; ++i) {
        const kdss_query &x = q[i];
        if (x.k < 2 || x.k > 255 || x.T < 0 || x.graph.n < 0 || x.graph.n >= (int64_t)INT32_MAX ||
            x.graph.m < 0 || x.graph.m > ((int64_t)1 << 30) ||
            (x.graph.m > 0 && (!x.graph.src || !x.graph.dst))) {
            status[i] = KDSS_ERR_INVALID_ARG;
            msgs[i] = "bad query: k in [2, 255], T >= 0, n in [0, 2^31 - 1), m in [0, 2^30], edge arrays";
            continue;
        }
        if (x.graph.on_device && x.graph.m > 0) {
            try {
                check_device_array(x.graph.src, (size_t)x.graph.m * sizeof(int32_t), "src");
                check_device_array(x.graph.dst, (size_t)x.graph.m * sizeof(int32_t), "dst");
            } catch (const Error &e) {
                status[i] = e.code;
                msgs[i] = e.msg;
                continue;
            }
        }
        Group &g = groups[{x.k, x.T}];
        g.k = x.k;
        g.T = x.T;
        g.members.push_back(i);
    }
    // union graphs and their SCTs
    std::vector<Group *> gl;
    int64_t n_all = 0, short_cap = 1;
    for (auto &kv : groups) {
        Group &g = kv.second;
        const int nm = (int)g.members.size();
        int64_t m = 0, hm = 0;
        std::vector<Member> mem(nm);
        for (int j = 0; j < nm; ++j) {
            const kdss_graph_desc &d = q[g.members[j]].graph;
            mem[j] = Member{d.src, d.dst, d.m, d.n, g.n, m};
            g.qbase.push_back(g.n);
            g.qn.push_back(d.n);
            g.n += d.n;
            m += d.m;
            if (!d.on_device) hm += d.m;
        }
        if (g.n >= (int64_t)INT32_MAX) fail(KDSS_ERR_UNSUPPORTED, "a batch group exceeds 2^31 - 1 nodes");
        if (m > ((int64_t)1 << 30)) fail(KDSS_ERR_UNSUPPORTED, "a batch group exceeds 2^30 edge records");
        DBuf<int32_t> us(c, m), ud(c, m), hs(c, hm), hd(c, hm);
        DBuf<int> bad(c, nm);
        zero(c, bad.p, bad.bytes());
        int64_t ho = 0;
        for (int j = 0; j < nm; ++j) {  // host edge lists: one staging copy each
            const kdss_graph_desc &d = q[g.members[j]].graph;
            if (d.on_device || d.m == 0) continue;
            to_device(c, hs.p + ho, d.src, d.m);
            to_device(c, hd.p + ho, d.dst, d.m);
            mem[j].src = hs.p + ho;
            mem[j].dst = hd.p + ho;
            ho += d.m;
        }
        if (m > 0) {
            DBuf<Member> dm(c, nm);
            to_device(c, dm.p, mem.data(), nm);
            k_union_edges<<<grid_for(c, m, 256, 4), 256, 0, c.stream>>>(dm.p, nm, m, us.p, ud.p, bad.p);
            KDSS_LAUNCH_CHECK();
            std::vector<int> hbad(nm);
            to_host(c, hbad.data(), bad.p, nm);  // synchronises: staging and table can go
            for (int j = 0; j < nm; ++j)
                if (hbad[j]) {
                    status[g.members[j]] = KDSS_ERR_BAD_GRAPH;
                    msgs[g.members[j]] = "an edge endpoint is outside [0, n)";
                }
        }
        kdss_graph_desc ud_desc{g.n, m, us.p, ud.p, 1};
        {
            GraphDev gd;
            build_graph(c, ud_desc, order, gd);
            build_sct(c, gd, g.k, g.s);
        }
        g.node_off = n_all;
        n_all += g.n;
        short_cap = std::max<int64_t>(short_cap, g.s.class_begin[3] - g.s.class_begin[0]);
        gl.push_back(&g);
    }
    if (gl.empty()) return;
    // exact range of the integer r, and of the prefix counts, per group
    for (Group *g : gl) {
        const long double lim = prec == KDSS_INT64 ? 9.2e18L : 9.007199254740992e15L;
        const long double ck = (long double)g->s.ck_lo + (long double)g->s.ck_hi * 18446744073709551616.0L;
        const char *why = nullptr;
        if (g->s.ck_hi) why = "prefix clique counts above 2^64 are not supported";
        else if (prec != KDSS_FP32K && (long double)g->T * ck >= lim) why = "T * c_k leaves the exact range of r";
        if (why) {
            for (int i : g->members) {
                status[i] = KDSS_ERR_OVERFLOW;
                msgs[i] = why;
            }
            g->T = 0;
            g->skip = true;
        }
    }
    // shared state; phases of equal active sets, each one CUDA graph replayed
    StateDev st;
    fw_init_n(c, n_all, short_cap, prec, st);
    std::vector<int> Ts;
    for (Group *g : gl) Ts.push_back(g->T);
    std::sort(Ts.begin(), Ts.end());
    Ts.erase(std::unique(Ts.begin(), Ts.end()), Ts.end());
    // Every iteration is one replayed CUDA graph: a work-queue pass over
    // every active group (k_pb_queue / k_pb_queue_f32 and the long-pair queue
    // kernels, `chunk` tiles per item), or the per-class kernels of each
    // group in turn (chunk 0), then the groups' steps.  The autotuner times
    // both forms on the run's own iterations.
    int chunk = opts ? opts->chunk : 0, tpp = opts ? opts->threads_per_path : 0;
    BatchTuning tune;
    int done = 0;
    for (int Tp : Ts) {
        if (Tp <= done) continue;
        std::vector<Group *> act;
        for (Group *g : gl) if (g->T >= Tp) act.push_back(g);
        std::vector<std::pair<const SctDev *, int64_t>> sets;
        for (Group *g : act) sets.push_back({&g->s, g->node_off});
        auto steps = [&](const Ctx &cc) {
            for (size_t j = 0; j < act.size(); ++j)
                fw_enqueue_step_range(cc, st, act[j]->node_off, act[j]->n, j + 1 == act.size());
        };
        auto run = [&](cudaGraphExec_t exec, long long nk, int iters, float *ms) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (ms) {
                KDSS_CUDA(cudaEventCreate(&e0));
                KDSS_CUDA(cudaEventCreate(&e1));
                KDSS_CUDA(cudaEventRecord(e0, c.stream));
            }
            cudaError_t e = cudaSuccess;
            for (int it = 0; it < iters && e == cudaSuccess; ++it) {
                e = cudaGraphLaunch(exec, c.stream);
                add_launches(nk);
            }
            check_cuda(e, "batch FW graph launch", __FILE__, __LINE__);
            if (ms) {
                KDSS_CUDA(cudaEventRecord(e1, c.stream));
                KDSS_CUDA(cudaEventSynchronize(e1));
                cudaEventElapsedTime(ms, e0, e1);
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
            }
        };
        auto graph_for = [&](int ch, int tp, QueuePlan &qp, cudaGraphExec_t *exec) {
            if (ch <= 0)
                return fw_capture(c, exec, [&](const Ctx &cc) {
                    for (Group *g : act) fw_enqueue_group(cc, g->s, st, g->node_off);
                    steps(cc);
                });
            queue_plan(c, sets, ch, tp, qp);
            return fw_capture(c, exec, [&](const Ctx &cc) {
                queue_enqueue(cc, qp, st);
                steps(cc);
            });
        };
        // autotuner: after two warm-up iterations, one iteration per candidate
        // (each is a real iteration of the run; the integer results do not
        // depend on the configuration, the FP32 ones only through the order
        // of their atomic sums), then the fastest for the rest
        if ((chunk <= 0 || tpp <= 0) && !tune.done) {
            std::vector<std::pair<int, int>> cand;
            bool has_long = false;
            for (Group *g : act) has_long |= g->s.class_begin[4] > g->s.class_begin[3];
            if (chunk <= 0 && (tpp <= 0 || tpp == 32)) cand.push_back({0, 32});   // per-class kernels
            for (int ch : {1, 4, 16})
                for (int tp : {32, 8})
                    if ((chunk <= 0 || ch == chunk) && (tpp <= 0 || tp == tpp) && (tp == 32 || has_long))
                        cand.push_back({ch, tp});
            const int warm = 2;
            if (Tp - done >= warm + (int)cand.size() + 1 && cand.size() > 1) {
                QueuePlan qp;
                cudaGraphExec_t exec = nullptr;
                long long nk = graph_for(4, 32, qp, &exec);
                run(exec, nk, warm, nullptr);
                cudaGraphExecDestroy(exec);
                done += warm;
                float best = 1e30f;
                for (auto &cf : cand) {
                    QueuePlan qc;
                    cudaGraphExec_t ex2 = nullptr;
                    nk = graph_for(cf.first, cf.second, qc, &ex2);
                    float ms = 0.f;
                    run(ex2, nk, 1, &ms);
                    cudaGraphExecDestroy(ex2);
                    ++done;
                    tune.tried.push_back({cf.first, cf.second, ms});
                    if (ms < best) { best = ms; tune.chunk = cf.first; tune.tpp = cf.second; }
                }
                tune.done = true;
            }
        }
        const int ch = chunk > 0 ? chunk : (tune.done ? tune.chunk : 4);
        const int tp = tpp > 0 ? tpp : (tune.done ? tune.tpp : 32);
        if (done < Tp) {
            QueuePlan qp;
            cudaGraphExec_t exec = nullptr;
            const long long nk = graph_for(ch, tp, qp, &exec);
            run(exec, nk, Tp - done, nullptr);
            cudaGraphExecDestroy(exec);
        }
        tune.chunk = ch;
        tune.tpp = tp;
        done = Tp;
    }
    set_last_batch_tuning(tune);
    int herr = 0;
    to_host(c, &herr, st.err.p, 1);
    if (herr) fail(KDSS_ERR_CUDA, "batch FW: water-filling invariant failed on the device");
    // extraction, segmented by query; every group reports its own T
    for (Group *g : gl) {
        if (g->skip) continue;
        st.t = g->T;
        extract_group(c, *g, st, out);
    }
    sync(c);
    for (int i = 0; i < nq; ++i) {
        if (status[i] != KDSS_OK) {
            free(out[i].ids);
            memset(&out[i], 0, sizeof out[i]);
        }
        out[i].status = status[i];
    }
}

}  // namespace kdss

extern "C" kdss_status kdss_batch_last_tuning(kdss_batch_tuning *out) {
    if (!out) return KDSS_ERR_INVALID_ARG;
    memset(out, 0, sizeof *out);
    const kdss::BatchTuning &t = kdss::last_batch_tuning();
    out->chunk = t.chunk;
    out->threads_per_path = t.tpp;
    out->autotuned = t.done ? 1 : 0;
    out->ntried = (int32_t)std::min<size_t>(t.tried.size(), 8);
    for (int i = 0; i < out->ntried; ++i) {
        out->tried_chunk[i] = t.tried[i].chunk;
        out->tried_threads_per_path[i] = t.tried[i].tpp;
        out->tried_ms[i] = t.tried[i].ms;
    }
    return KDSS_OK;
}
