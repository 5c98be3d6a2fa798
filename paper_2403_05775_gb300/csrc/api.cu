// api.cu -- the extern "C" entry points declared in include/kdss.h.
//
// Every entry point converts internal exceptions into a kdss_status and a
// thread-local message; nothing throws across the boundary.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fw.cuh"

#include "handles.cuh"

using namespace kdss;

namespace kdss {
void extract_prefix(const Ctx &c, const SctDev &s, const StateDev &st, kdss_result *out);
void solve_streamed(const Ctx &c, const kdss_graph_desc &g, int k, int T, int nchunks, int precision,
                    int order, kdss_result *out);
void solve_batch(const kdss_query *q, int nq, kdss_result *out, const kdss_opts *opts,
                 std::vector<kdss_status> &status, std::vector<std::string> &msgs);
void cpsample_run(const Ctx &c, const kdss_graph_desc &g, int k, int64_t t, int T, uint64_t seed,
                  int order, kdss_result *out, kdss_cpsample_stats *stats);
}

namespace {

thread_local std::string g_last_error;

kdss_status record(kdss_status code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

}  // namespace

namespace kdss {
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace kdss

namespace {

#define API_BEGIN \
    try {         \
        g_last_error.clear();
#define API_END                                                                  \
    }                                                                            \
    catch (const kdss::Error &e) { return record(e.code, e.msg); }               \
    catch (const std::bad_alloc &) { return record(KDSS_ERR_OOM, "host allocation failed"); } \
    catch (const std::exception &e) { return record(KDSS_ERR_CUDA, e.what()); }  \
    catch (...) { return record(KDSS_ERR_CUDA, "unknown internal error"); }      \
    return KDSS_OK;

void check_graph(const kdss_graph_desc *g) {
    if (!g) fail(KDSS_ERR_INVALID_ARG, "graph descriptor is NULL");
    if (g->n < 0 || g->n >= (int64_t)INT32_MAX) fail(KDSS_ERR_INVALID_ARG, "n must be in [0, 2^31 - 1)");
    if (g->m < 0) fail(KDSS_ERR_INVALID_ARG, "m must be >= 0");
    if (g->m > 0 && (!g->src || !g->dst)) fail(KDSS_ERR_INVALID_ARG, "edge arrays are NULL");
    if (g->m > ((int64_t)1 << 30)) fail(KDSS_ERR_UNSUPPORTED, "more than 2^30 edge records");
    if (g->on_device && g->m > 0) {
        check_device_array(g->src, (size_t)g->m * sizeof(int32_t), "src");
        check_device_array(g->dst, (size_t)g->m * sizeof(int32_t), "dst");
    }
}

void check_k(int32_t k) {
    if (k < 2 || k > 255) fail(KDSS_ERR_INVALID_ARG, "k must be in [2, 255]");
}

int64_t sct_bytes(const kdss_sct *h) {
    const GraphDev &g = h->g;
    const SctDev &s = h->s;
    return (int64_t)(g.off.bytes() + g.adj.bytes() + g.core.bytes() + g.rnd.bytes() +
                     g.rank.bytes() + g.vert.bytes() + g.out_off.bytes() + g.out_adj.bytes() +
                     s.pair_off.bytes() + s.nodes.bytes() + s.h.bytes() + binom_bytes(s) +
                     (h->shared ? h->fc.bytes() : 0));
}

// Calls that need the flat pairs refuse the prefix-shared form.
void require_flat(const kdss_sct *s) {
    if (s->shared)
        fail(KDSS_ERR_INVALID_ARG,
             "a prefix-shared SCT: this call needs the flat pairs (keep the handle it was made from)");
}

kdss_status build_impl(const kdss_graph_desc *g, int32_t k, const kdss_opts *opts, kdss_sct **out,
                       int klo = -1) {
    API_BEGIN
    if (!out) fail(KDSS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    check_graph(g);
    check_k(k);
    const int order = opts ? opts->order : KDSS_ORDER_PEEL;
    if (order != KDSS_ORDER_PEEL && order != KDSS_ORDER_CORE)
        fail(KDSS_ERR_INVALID_ARG, "unknown vertex order");
    Ctx c = make_ctx(opts);
    kdss_sct *h = new kdss_sct();
    try {
        h->ctx = c;
        build_graph(c, *g, order, h->g);
        build_sct(c, h->g, k, h->s, klo);
        if (klo >= 0 && klo < k) h->kmax_multi = k;
        h->m = h->g.nadj / 2;
        h->degeneracy = h->g.degeneracy;
        h->max_out = h->g.max_out;
        h->has_graph = true;
        if (!(opts && (opts->flags & KDSS_FLAG_KEEP_GRAPH))) {
            h->g.off.reset(); h->g.adj.reset(); h->g.core.reset(); h->g.rnd.reset();
            h->g.rank.reset(); h->g.vert.reset(); h->g.out_off.reset(); h->g.out_adj.reset();
            h->has_graph = false;
        }
        sync(c);
    } catch (...) {
        delete h;
        throw;
    }
    *out = h;
    API_END
}

kdss_status batch_impl(const kdss_query *q, int32_t nq, kdss_result *out, const kdss_opts *opts,
                       std::vector<kdss_status> &status, std::vector<std::string> &msgs) {
    API_BEGIN
    const int order = opts ? opts->order : KDSS_ORDER_PEEL;
    if (order != KDSS_ORDER_PEEL && order != KDSS_ORDER_CORE)
        fail(KDSS_ERR_INVALID_ARG, "unknown vertex order");
    solve_batch(q, nq, out, opts, status, msgs);
    API_END
}

}  // namespace

extern "C" {

kdss_status kdss_build_sct(const kdss_graph_desc *g, int32_t k, const kdss_opts *opts,
                           kdss_sct **out) {
    return build_impl(g, k, opts, out);
}

kdss_status kdss_build_sct_multi(const kdss_graph_desc *g, int32_t k_max, const kdss_opts *opts,
                                 kdss_sct **out) {
    return build_impl(g, k_max, opts, out, 2);
}

kdss_status kdss_sct_restrict(const kdss_sct *multi, int32_t k, const kdss_opts *opts,
                              kdss_sct **out) {
    API_BEGIN
    if (!multi || !out) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    require_flat(multi);
    if (multi->kmax_multi <= 0) fail(KDSS_ERR_INVALID_ARG, "not a k-agnostic SCT (kdss_build_sct_multi)");
    if (k < 2 || k > multi->kmax_multi) fail(KDSS_ERR_INVALID_ARG, "k must be in [2, k_max of the SCT]");
    Ctx c = make_ctx(opts);
    kdss_sct *h = new kdss_sct();
    try {
        h->ctx = c;
        sct_restrict(c, multi->s, k, h->s);
        h->m = multi->m;
        h->degeneracy = multi->degeneracy;
        h->max_out = multi->max_out;
        sync(c);
    } catch (...) {
        delete h;
        throw;
    }
    *out = h;
    API_END
}

kdss_status kdss_solve_streamed(const kdss_graph_desc *g, int32_t k, int32_t T, int32_t nchunks,
                                const kdss_opts *opts, kdss_result *out) {
    API_BEGIN
    if (!out) fail(KDSS_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof *out);
    check_graph(g);
    check_k(k);
    if (T < 0) fail(KDSS_ERR_INVALID_ARG, "T must be >= 0");
    if (nchunks < 1) fail(KDSS_ERR_INVALID_ARG, "nchunks must be >= 1");
    const int prec = opts ? opts->precision : KDSS_INT64;
    if (prec != KDSS_INT64 && prec != KDSS_FP64 && prec != KDSS_FP32K)
        fail(KDSS_ERR_INVALID_ARG, "unknown precision");
    if (opts && (opts->flags & KDSS_FLAG_ASYNC))
        fail(KDSS_ERR_UNSUPPORTED, "the streamed solve runs the synchronous iterations only");
    const int order = opts ? opts->order : KDSS_ORDER_PEEL;
    if (order != KDSS_ORDER_PEEL && order != KDSS_ORDER_CORE)
        fail(KDSS_ERR_INVALID_ARG, "unknown vertex order");
    Ctx c = make_ctx(opts);
    solve_streamed(c, *g, k, T, nchunks, prec, order, out);
    sync(c);
    API_END
}

kdss_status kdss_sct_count(const kdss_graph_desc *g, int32_t k, double budget_s,
                           const kdss_opts *opts, kdss_sct_count_stats *out) {
    API_BEGIN
    if (!out) fail(KDSS_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof *out);
    check_graph(g);
    check_k(k);
    if (!(budget_s >= 0)) fail(KDSS_ERR_INVALID_ARG, "budget_s must be >= 0");
    const int order = opts ? opts->order : KDSS_ORDER_PEEL;
    if (order != KDSS_ORDER_PEEL && order != KDSS_ORDER_CORE)
        fail(KDSS_ERR_INVALID_ARG, "unknown vertex order");
    Ctx c = make_ctx(opts);
    GraphDev gd;
    build_graph(c, *g, order, gd);
    out->m = gd.nadj / 2;
    out->degeneracy = gd.degeneracy;
    out->max_out_degree = gd.max_out;
    gd.off.reset();
    gd.adj.reset();
    SctCount sc;
    count_sct(c, gd, k, budget_s, sc);
    out->eta_k = sc.eta;
    out->L_k = sc.L;
    out->c_k_lo = sc.ck_lo;
    out->c_k_hi = sc.ck_hi;
    for (int cl = 0; cl <= NCLASS; ++cl) out->pairs_per_class[cl] = sc.pairs_per_class[cl];
    out->roots_total = sc.roots_total;
    out->roots_done = sc.roots_done;
    out->roots_cut = sc.roots_cut;
    out->cut_pairs = sc.cut_pairs;
    out->cut_nodes = sc.cut_nodes;
    out->complete = sc.complete;
    out->max_pair_len = sc.max_len;
    out->count_bits = sc.count_bits;
    out->seconds = sc.seconds;
    sync(c);
    API_END
}

kdss_status kdss_sct_from_pairs(int64_t n, int32_t k, int64_t npairs, const int64_t *pair_off,
                                const int32_t *nodes, const int32_t *h, int32_t on_device,
                                const kdss_opts *opts, kdss_sct **out) {
    API_BEGIN
    if (!out) fail(KDSS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    check_k(k);
    if (n < 0 || n >= (int64_t)INT32_MAX) fail(KDSS_ERR_INVALID_ARG, "n must be in [0, 2^31 - 1)");
    if (npairs < 0 || npairs >= (int64_t)INT32_MAX) fail(KDSS_ERR_INVALID_ARG, "npairs out of range");
    if (npairs > 0 && (!pair_off || !nodes || !h)) fail(KDSS_ERR_INVALID_ARG, "pair arrays are NULL");
    Ctx c = make_ctx(opts);
    kdss_sct *hd = new kdss_sct();
    try {
        hd->ctx = c;
        DBuf<int64_t> doff;
        DBuf<int32_t> dnodes, dh;
        const int64_t *po = pair_off;
        const int32_t *pn = nodes, *ph = h;
        int64_t nn = 0;
        if (npairs > 0) {
            if (on_device) {
                check_device_array(pair_off, (size_t)(npairs + 1) * sizeof(int64_t), "pair_off");
                check_device_array(h, (size_t)npairs * sizeof(int32_t), "h");
                to_host(c, &nn, pair_off + npairs, 1);
                if (nn < 0) fail(KDSS_ERR_INVALID_ARG, "pair_off[npairs] must be >= 0");
                check_device_array(nodes, (size_t)nn * sizeof(int32_t), "nodes");
            } else {
                nn = pair_off[npairs];
                if (pair_off[0] != 0) fail(KDSS_ERR_INVALID_ARG, "pair_off[0] must be 0");
                for (int64_t q = 0; q < npairs; ++q)
                    if (pair_off[q + 1] < pair_off[q]) fail(KDSS_ERR_INVALID_ARG, "pair_off must be non-decreasing");
                doff = DBuf<int64_t>(c, (size_t)npairs + 1);
                dnodes = DBuf<int32_t>(c, (size_t)std::max<int64_t>(nn, 1));
                dh = DBuf<int32_t>(c, (size_t)npairs);
                to_device(c, doff.p, pair_off, (size_t)npairs + 1);
                to_device(c, dnodes.p, nodes, (size_t)nn);
                to_device(c, dh.p, h, (size_t)npairs);
                po = doff.p; pn = dnodes.p; ph = dh.p;
            }
        }
        sct_from_pairs(c, n, k, npairs, po, pn, ph, hd->s);
        sync(c);
    } catch (...) {
        delete hd;
        throw;
    }
    *out = hd;
    API_END
}

kdss_status kdss_sct_info(const kdss_sct *s, kdss_sct_stats *out) {
    API_BEGIN
    if (!s || !out) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
    memset(out, 0, sizeof *out);
    out->n = s->s.n;
    out->m = s->m;
    out->eta_k = s->s.npairs;
    out->L_k = s->s.nnodes;
    out->c_k_lo = s->s.ck_lo;
    out->c_k_hi = s->s.ck_hi;
    out->k = s->s.k;
    out->degeneracy = s->degeneracy;
    out->max_out_degree = s->max_out;
    out->max_pair_len = s->s.max_len;
    out->device_bytes = sct_bytes(s);
    for (int c = 0; c < NCLASS && c < 8; ++c)
        out->pairs_per_class[c] = s->s.class_begin[c + 1] - s->s.class_begin[c];
    API_END
}

kdss_status kdss_sct_copy_pairs(const kdss_sct *s, int64_t *pair_off, int32_t *nodes, int32_t *h) {
    API_BEGIN
    if (!s) fail(KDSS_ERR_INVALID_ARG, "NULL handle");
    const Ctx &c = s->ctx;
    SctDev dec;
    if (s->shared) fc_decode_all(c, s->s, s->fc, dec);   // the pairs in the shared order
    const SctDev &f = s->shared ? dec : s->s;
    if (pair_off) to_host(c, pair_off, f.pair_off.p, (size_t)s->s.npairs + 1);
    if (nodes) to_host(c, nodes, f.nodes.p, (size_t)s->s.nnodes);
    if (h && s->s.npairs > 0) {
        std::vector<uint8_t> tmp((size_t)s->s.npairs);
        to_host(c, tmp.data(), f.h.p, tmp.size());
        for (size_t i = 0; i < tmp.size(); ++i) h[i] = tmp[i];
    }
    API_END
}

kdss_status kdss_sct_copy_graph(const kdss_sct *s, int64_t *off, int32_t *adj, int32_t *core,
                                int32_t *round_, int32_t *rank) {
    API_BEGIN
    if (!s) fail(KDSS_ERR_INVALID_ARG, "NULL handle");
    if (!s->has_graph) fail(KDSS_ERR_INVALID_ARG, "the handle keeps no graph (build with KDSS_FLAG_KEEP_GRAPH)");
    const Ctx &c = s->ctx;
    const GraphDev &g = s->g;
    if (off) to_host(c, off, g.off.p, (size_t)g.n + 1);
    if (adj) to_host(c, adj, g.adj.p, (size_t)g.nadj);
    if (core) to_host(c, core, g.core.p, (size_t)g.n);
    if (round_) to_host(c, round_, g.rnd.p, (size_t)g.n);
    if (rank) to_host(c, rank, g.rank.p, (size_t)g.n);
    API_END
}

namespace {
kdss_status fw_iterate_impl(kdss_sct *s, int32_t k, kdss_state **state, int32_t T,
                            const kdss_opts *opts) {
    API_BEGIN
    if (!s || !state) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
    if (k < 0 && s->kmax_multi)
        fail(KDSS_ERR_INVALID_ARG, "a k-agnostic SCT: name the k (kdss_fw_iterate_at) or restrict it");
    if (k >= 0) {
        const int kmax = s->kmax_multi ? s->kmax_multi : s->s.k;
        if (k < 2 || k > kmax || (!s->kmax_multi && k != s->s.k))
            fail(KDSS_ERR_INVALID_ARG, "k outside the P_k the SCT holds");
    }
    if (T < 0) fail(KDSS_ERR_INVALID_ARG, "T must be >= 0");
    if (*state && k >= 0 && (*state)->st.k != k)
        fail(KDSS_ERR_INVALID_ARG, "the state iterates another k");
    Ctx c = make_ctx(opts);
    if (s->shared && opts && ((opts->flags & KDSS_FLAG_ASYNC) || opts->chunk > 0))
        fail(KDSS_ERR_UNSUPPORTED,
             "a prefix-shared SCT iterates in the synchronous form on the per-class kernels "
             "(no KDSS_FLAG_ASYNC, no work-queue chunk)");
    bool created = false;
    if (!*state) {
        const int prec = opts ? opts->precision : KDSS_INT64;
        if (prec != KDSS_INT64 && prec != KDSS_FP64 && prec != KDSS_FP32K)
            fail(KDSS_ERR_INVALID_ARG, "unknown precision");
        kdss_state *st = new kdss_state();
        if (opts && opts->chunk > 0) {
            st->st.qchunk = opts->chunk;
            st->st.qtpp = opts->threads_per_path == 8 ? 8 : 32;
        }
        st->st.force_rooted = opts && (opts->flags & KDSS_FLAG_ROOTED);
        try {
            if (s->shared) fc_state_init(c, s->s, s->fc, k < 0 ? s->s.k : k, prec, st->st);
            else fw_init(c, s->s, prec, st->st, k);
        } catch (...) {
            delete st;
            throw;
        }
        *state = st;
        created = true;
    }
    if ((*state)->st.n != s->s.n) fail(KDSS_ERR_INVALID_ARG, "state and SCT differ in n");
    (*state)->st.per_iteration = opts && (opts->flags & KDSS_FLAG_PER_ITERATION);
    try {
        if (s->shared)
            fc_iterate(c, s->s, s->fc, (*state)->st, T, opts && (opts->flags & KDSS_FLAG_PROFILE));
        else if (opts && (opts->flags & KDSS_FLAG_ASYNC))
            fw_run_async(c, s->s, (*state)->st, T);
        else
            fw_run(c, s->s, (*state)->st, T, opts && (opts->flags & KDSS_FLAG_PROFILE));
        sync(c);
    } catch (...) {
        if (created) { delete *state; *state = nullptr; }
        throw;
    }
    API_END
}
}  // namespace

kdss_status kdss_fw_iterate(kdss_sct *s, kdss_state **state, int32_t T, const kdss_opts *opts) {
    return fw_iterate_impl(s, -1, state, T, opts);
}

kdss_status kdss_fw_iterate_at(kdss_sct *s, int32_t k, kdss_state **state, int32_t T,
                               const kdss_opts *opts) {
    return fw_iterate_impl(s, k, state, T, opts);
}

kdss_status kdss_sct_copy_cliques(kdss_sct *s, int32_t *cliques, int64_t capacity,
                                  int64_t *count) {
    API_BEGIN
    if (!s || !count) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
    require_flat(s);
    if (s->kmax_multi) fail(KDSS_ERR_INVALID_ARG, "a k-agnostic SCT: restrict it to one k first");
    if (capacity < 0 || (capacity > 0 && !cliques)) fail(KDSS_ERR_INVALID_ARG, "bad output buffer");
    if (s->nclq < 0) expand_cliques(s->ctx, s->s, s->cliques, s->nclq);
    *count = s->nclq;
    const int64_t rows = std::min<int64_t>(capacity, s->nclq);
    if (rows > 0) to_host(s->ctx, cliques, s->cliques.p, (size_t)(rows * s->s.k));
    API_END
}

kdss_status kdss_fw_cliques(kdss_sct *s, kdss_state **state, int32_t T, const kdss_opts *opts) {
    API_BEGIN
    if (!s || !state) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
    require_flat(s);
    if (s->kmax_multi) fail(KDSS_ERR_INVALID_ARG, "a k-agnostic SCT: restrict it to one k first");
    if (T < 0) fail(KDSS_ERR_INVALID_ARG, "T must be >= 0");
    Ctx c = make_ctx(opts);
    if (s->nclq < 0) expand_cliques(s->ctx, s->s, s->cliques, s->nclq);
    bool created = false;
    if (!*state) {
        const int prec = opts ? opts->precision : KDSS_INT64;
        if (prec != KDSS_INT64) fail(KDSS_ERR_UNSUPPORTED, "Alg. 1 iterations keep r in KDSS_INT64");
        kdss_state *st = new kdss_state();
        try {
            fw_init(c, s->s, prec, st->st);
        } catch (...) {
            delete st;
            throw;
        }
        *state = st;
        created = true;
    }
    if ((*state)->st.n != s->s.n) fail(KDSS_ERR_INVALID_ARG, "state and SCT differ in n");
    try {
        fw_cliques_run(c, s->cliques.p, s->nclq, s->s.k, (*state)->st, T);
        sync(c);
    } catch (...) {
        if (created) { delete *state; *state = nullptr; }
        throw;
    }
    API_END
}

kdss_status kdss_cpsample(const kdss_graph_desc *g, int32_t k, int64_t t, int32_t T, uint64_t seed,
                          const kdss_opts *opts, kdss_result *out, kdss_cpsample_stats *stats) {
    API_BEGIN
    if (!out) fail(KDSS_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof *out);
    check_graph(g);
    const int order = opts ? opts->order : KDSS_ORDER_PEEL;
    if (order != KDSS_ORDER_PEEL && order != KDSS_ORDER_CORE)
        fail(KDSS_ERR_INVALID_ARG, "unknown vertex order");
    Ctx c = make_ctx(opts);
    try {
        cpsample_run(c, *g, k, t, T, seed, order, out, stats);
    } catch (...) {
        free(out->ids);
        memset(out, 0, sizeof *out);
        throw;
    }
    API_END
}

kdss_status kdss_state_copy_r(const kdss_state *st, void *r_host, int32_t *t_out) {
    API_BEGIN
    if (!st) fail(KDSS_ERR_INVALID_ARG, "NULL state");
    const StateDev &d = st->st;
    if (r_host) {
        if (d.precision == KDSS_FP32K) to_host(d.ctx, (float *)r_host, d.r32.p, (size_t)d.n);
        else to_host(d.ctx, (uint64_t *)r_host, d.r.p, (size_t)d.n);
    }
    if (t_out) *t_out = d.t;
    API_END
}

kdss_status kdss_state_timing(const kdss_state *st, kdss_timing *out) {
    API_BEGIN
    if (!st || !out) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
    *out = st->st.timing;
    API_END
}

kdss_status kdss_extract(const kdss_sct *s, const kdss_state *st, const kdss_opts *opts,
                         kdss_result *out) {
    API_BEGIN
    if (!s || !st || !out) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
    if (st->st.n != s->s.n) fail(KDSS_ERR_INVALID_ARG, "state and SCT differ in n");
    if (st->st.k < 2 || st->st.k > s->s.k) fail(KDSS_ERR_INVALID_ARG, "the state's k is not in the SCT");
    Ctx c = make_ctx(opts);
    if (s->shared) fc_extract(c, s->s, s->fc, st->st, out);
    else extract_prefix(c, s->s, st->st, out);
    API_END
}

kdss_status kdss_sct_share_prefixes(const kdss_sct *in, int64_t chunk_pairs, const kdss_opts *opts,
                                    kdss_sct **out) {
    API_BEGIN
    if (!in || !out) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    require_flat(in);
    if (chunk_pairs < 0) fail(KDSS_ERR_INVALID_ARG, "chunk_pairs must be >= 0");
    Ctx c = make_ctx(opts);
    kdss_sct *h = new kdss_sct();
    try {
        h->ctx = c;
        const SctDev &f = in->s;
        SctDev &m = h->s;
        m.k = f.k;
        m.n = f.n;
        m.npairs = f.npairs;
        m.nnodes = f.nnodes;
        for (int cl = 0; cl <= NCLASS; ++cl) m.class_begin[cl] = f.class_begin[cl];
        m.ck_lo = f.ck_lo;
        m.ck_hi = f.ck_hi;
        m.max_len = f.max_len;
        m.binom = DBuf<uint64_t>(c, f.binom.n);
        m.binom128 = DBuf<U128>(c, f.binom128.n);
        m.binomf = DBuf<float>(c, f.binomf.n);
        if (f.binom.n)
            KDSS_CUDA(cudaMemcpyAsync(m.binom.p, f.binom.p, f.binom.bytes(), cudaMemcpyDeviceToDevice, c.stream));
        if (f.binom128.n)
            KDSS_CUDA(cudaMemcpyAsync(m.binom128.p, f.binom128.p, f.binom128.bytes(),
                                      cudaMemcpyDeviceToDevice, c.stream));
        if (f.binomf.n)
            KDSS_CUDA(cudaMemcpyAsync(m.binomf.p, f.binomf.p, f.binomf.bytes(), cudaMemcpyDeviceToDevice,
                                      c.stream));
        m.binom_rows = f.binom_rows;
        fc_encode(c, f, chunk_pairs > 0 ? chunk_pairs : (int64_t)1 << 22, h->fc);
        h->shared = true;
        h->m = in->m;
        h->degeneracy = in->degeneracy;
        h->max_out = in->max_out;
        h->kmax_multi = in->kmax_multi;
        sync(c);
    } catch (...) {
        delete h;
        throw;
    }
    *out = h;
    API_END
}

kdss_status kdss_sct_shared_words(const kdss_sct *s, int64_t *words, int64_t *chunks) {
    API_BEGIN
    if (!s) fail(KDSS_ERR_INVALID_ARG, "NULL handle");
    if (!s->shared) fail(KDSS_ERR_INVALID_ARG, "not a prefix-shared SCT (kdss_sct_share_prefixes)");
    if (words) *words = s->fc.nwords;
    if (chunks) *chunks = (int64_t)s->fc.chunks.size();
    API_END
}

kdss_status kdss_solve(const kdss_graph_desc *g, int32_t k, int32_t T, const kdss_opts *opts,
                       kdss_result *out) {
    if (!out) return record(KDSS_ERR_INVALID_ARG, "out is NULL");
    memset(out, 0, sizeof *out);
    kdss_sct *s = nullptr;
    kdss_state *st = nullptr;
    kdss_status rc = kdss_build_sct(g, k, opts, &s);
    const int32_t every = opts ? opts->check_every : 0;
    const double eps = opts ? opts->eps_stop : 0.0;
    if (rc == KDSS_OK && every > 0 && eps > 0.0 && T > 0) {
        // stop rule: the certificate gap after every `every` iterations
        int32_t t = 0;
        while (rc == KDSS_OK && t < T) {
            const int32_t j = std::min(every, T - t);
            rc = kdss_fw_iterate(s, &st, j, opts);
            t += j;
            if (rc != KDSS_OK || t >= T) break;
            kdss_result chk;
            memset(&chk, 0, sizeof chk);
            rc = kdss_extract(s, st, opts, &chk);
            const bool stop = rc == KDSS_OK && chk.gap <= eps;
            kdss_result_free(&chk);
            if (stop) break;
        }
    } else if (rc == KDSS_OK) {
        rc = kdss_fw_iterate(s, &st, T, opts);
    }
    if (rc == KDSS_OK) rc = kdss_extract(s, st, opts, out);
    if (rc == KDSS_OK) out->T = T;
    out->status = rc;
    std::string msg = g_last_error;
    kdss_state_free(st);
    kdss_sct_free(s);
    g_last_error = msg;
    return rc;
}

kdss_status kdss_solve_batch(const kdss_query *q, int32_t nq, kdss_result *out,
                             const kdss_opts *opts) {
    if (nq < 0 || (nq > 0 && (!q || !out))) return record(KDSS_ERR_INVALID_ARG, "bad batch arguments");
    for (int32_t i = 0; i < nq; ++i) memset(&out[i], 0, sizeof out[i]);
    std::vector<kdss_status> status;
    std::vector<std::string> msgs;
    const kdss_status rc = batch_impl(q, nq, out, opts, status, msgs);
    if (rc != KDSS_OK) {  // the whole batch failed: every query carries its status
        for (int32_t i = 0; i < nq; ++i) {
            free(out[i].ids);
            memset(&out[i], 0, sizeof out[i]);
            out[i].status = rc;
        }
        return rc;
    }
    for (int32_t i = 0; i < nq; ++i)
        if (status[i] != KDSS_OK) return record(status[i], msgs[i]);
    return record(KDSS_OK, "");
}

void kdss_sct_free(kdss_sct *s) {
    if (!s) return;
    cudaStreamSynchronize(s->ctx.stream);
    delete s;
}

void kdss_state_free(kdss_state *st) {
    if (!st) return;
    cudaStreamSynchronize(st->st.ctx.stream);
    delete st;
}

void kdss_result_free(kdss_result *r) {
    if (!r) return;
    free(r->ids);
    r->ids = nullptr;
}

const char *kdss_last_error(void) { return g_last_error.c_str(); }

const char *kdss_version(void) { return "kdss-gb300 0.1 (sm_103a)"; }

int64_t kdss_kernel_launches(void) { return (int64_t)kdss::launches(); }

}  // extern "C"
