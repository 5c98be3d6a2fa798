// server.cu -- continuous-batching query server (include/kdss_server.h).
//
// Two host threads share a query table under one mutex:
//   builder  : pending queue (arrival order) -> SCT build on the build stream,
//              admitted while the resident bytes are below the budget;
//   iterator : built queries join the active set; each round replays one CUDA
//              graph that runs one FW iteration of every active query (the
//              PBUpdate launches of each query's SCT on its own state, then
//              each state's step); the graph is captured again only when the
//              active set changes.  The round length is the smallest distance
//              of an active query to its next stop check, so every query is
//              checked after exactly check_every of its own iterations, as
//              kdss_solve does.
// Device memory of a finished query is released on the build stream after
// the iterator has synchronised its own stream (the extraction reads back).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "handles.cuh"
#include "kdss_server.h"

namespace kdss {
void extract_prefix(const Ctx &c, const SctDev &s, const StateDev &st, kdss_result *out);
void set_last_error(const std::string &msg);
}  // namespace kdss

using namespace kdss;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

enum class QState { Pending, Building, Built, Active, Done };

struct Query {
    int64_t ticket = 0;
    int k = 0, T = 0;
    int64_t n = 0, m = 0;
    std::vector<int32_t> hsrc, hdst;  // host edge list (host submissions)
    DBuf<int32_t> dsrc, ddst;         // device copy (device submissions)
    QState state = QState::Pending;
    std::unique_ptr<kdss_sct> sct;
    std::unique_ptr<StateDev> st;
    int64_t bytes = 0;
    int peak_batch = 0;
    int checked_at = -1;  // iteration count of the last stop check
    Clock::time_point t_submit, t_build0, t_built, t_first, t_done;
    kdss_result res{};
    kdss_status status = KDSS_OK;
    std::string msg;
};

int64_t sct_footprint(const SctDev &s) {
    return (int64_t)(s.pair_off.bytes() + s.nodes.bytes() + s.h.bytes() + binom_bytes(s));
}

int64_t state_footprint(const SctDev &s, int precision) {
    const int64_t n = std::max<int64_t>(s.n, 1);
    // r and delta (8 + 8 bytes), or r, compensation, allocation and its
    // error terms (4 x 4 bytes); the list of pairs left to the slow kernel
    (void)precision;
    return n * 16 + 4 * std::max<int64_t>(1, s.class_begin[3] - s.class_begin[0]) + 64;
}

}  // namespace

struct kdss_server {
    kdss_server_opts o{};
    int device = 0;
    Ctx bctx, wctx;  // build stream, iteration stream
    cudaStream_t bstream = nullptr, wstream = nullptr;
    std::mutex mu;
    std::condition_variable cv_build, cv_iter, cv_done;
    std::unordered_map<int64_t, std::unique_ptr<Query>> table;
    std::deque<Query *> pending;
    std::vector<Query *> built;  // waiting for the iterator
    int64_t next_ticket = 1;
    int64_t resident = 0, peak_resident = 0;
    int64_t submitted = 0, completed = 0, failed = 0, replays = 0, captures = 0;
    int peak_active = 0;
    int active_count = 0;
    bool stop = false;
    std::thread builder, iterator;

    void finish(Query *q, kdss_status st, const std::string &m);  // holds mu
    void build_loop();
    void iterate_loop();
};

void kdss_server::finish(Query *q, kdss_status st, const std::string &m) {
    q->status = st;
    q->msg = m;
    q->t_done = Clock::now();
    q->state = QState::Done;
    if (st == KDSS_OK) ++completed; else ++failed;
    cv_done.notify_all();
}

void kdss_server::build_loop() {
    cudaSetDevice(device);
    while (true) {
        Query *q = nullptr;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_build.wait(lk, [&] {
                return stop || (!pending.empty() && (resident < o.hbm_budget || resident == 0));
            });
            if (stop) return;
            q = pending.front();
            pending.pop_front();
            q->state = QState::Building;
            q->t_build0 = Clock::now();
        }
        kdss_status st = KDSS_OK;
        std::string msg;
        std::unique_ptr<kdss_sct> h;
        try {
            h.reset(new kdss_sct());
            h->ctx = bctx;
            kdss_graph_desc g{q->n, q->m, nullptr, nullptr, 0};
            if (q->dsrc.p) { g.src = q->dsrc.p; g.dst = q->ddst.p; g.on_device = 1; }
            else { g.src = q->hsrc.data(); g.dst = q->hdst.data(); }
            build_graph(bctx, g, o.order, h->g);
            build_sct(bctx, h->g, q->k, h->s);
            h->m = h->g.nadj / 2;
            h->degeneracy = h->g.degeneracy;
            h->max_out = h->g.max_out;
            h->g = GraphDev();  // the CSR is not needed for the iterations
            h->has_graph = false;
            sync(bctx);
            q->dsrc.reset();
            q->ddst.reset();
            std::vector<int32_t>().swap(q->hsrc);
            std::vector<int32_t>().swap(q->hdst);
        } catch (const Error &e) {
            st = e.code;
            msg = e.msg;
        } catch (const std::bad_alloc &) {
            st = KDSS_ERR_OOM;
            msg = "host allocation failed";
        }
        std::unique_lock<std::mutex> lk(mu);
        if (st == KDSS_OK) {
            q->sct = std::move(h);
            q->bytes = sct_footprint(q->sct->s) + state_footprint(q->sct->s, o.precision);
            resident += q->bytes;
            peak_resident = std::max(peak_resident, resident);
            q->t_built = Clock::now();
            q->state = QState::Built;
            built.push_back(q);
            cv_iter.notify_all();
        } else if (st == KDSS_ERR_OOM && resident > 0) {
            // wait for memory: back to the head of the queue until a query
            // that holds memory finishes
            h.reset();
            q->state = QState::Pending;
            pending.push_front(q);
            const int64_t held = resident;
            cv_build.wait(lk, [&] { return stop || resident < held; });
        } else {
            finish(q, st, msg);
        }
    }
}

void kdss_server::iterate_loop() {
    cudaSetDevice(device);
    std::vector<Query *> active;
    cudaGraphExec_t exec = nullptr;
    long long nk = 0;
    bool dirty = true;
    const int every = o.check_every;
    const bool inplace = (o.flags & KDSS_FLAG_ASYNC) != 0;
    auto drop_exec = [&] {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
    };
    while (true) {
        std::vector<Query *> joined;
        {
            std::unique_lock<std::mutex> lk(mu);
            cv_iter.wait(lk, [&] { return stop || !built.empty() || !active.empty(); });
            if (stop) break;
            while (!built.empty() && (int)active.size() + (int)joined.size() < o.max_active) {
                joined.push_back(built.front());
                built.erase(built.begin());
            }
        }
        try {
            for (Query *q : joined) active.push_back(q);  // finished on any error below
            for (Query *q : joined) {
                q->st.reset(new StateDev());
                fw_init(wctx, q->sct->s, o.precision, *q->st);
                q->t_first = Clock::now();
                dirty = true;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                active_count = (int)active.size();
                peak_active = std::max(peak_active, active_count);
                for (Query *q : active) q->peak_batch = std::max(q->peak_batch, active_count);
            }
            // round length: the nearest stop check of any active query
            int j = every;
            for (Query *q : active) {
                const int t = q->st->t;
                j = std::min(j, std::min(every - t % every, q->T - t));
            }
            if (j > 0) {
                if (dirty) {
                    drop_exec();
                    nk = fw_capture(wctx, &exec, [&](const Ctx &cc) {
                        for (Query *q : active) {
                            if (inplace) {
                                fw_enqueue_inplace(cc, q->sct->s, *q->st);
                            } else {
                                fw_enqueue_group(cc, q->sct->s, *q->st, 0);
                                fw_enqueue_step_range(cc, *q->st, 0, q->sct->s.n, true);
                            }
                        }
                    });
                    dirty = false;
                    std::lock_guard<std::mutex> lk(mu);
                    ++captures;
                }
                for (int it = 0; it < j; ++it) {
                    KDSS_CUDA(cudaGraphLaunch(exec, wctx.stream));
                    add_launches(nk);
                }
                for (Query *q : active) q->st->t += j;
                std::lock_guard<std::mutex> lk(mu);
                replays += j;
            }
            sync(wctx);
            // stop checks
            std::vector<Query *> keep;
            for (Query *q : active) {
                const int t = q->st->t;
                const bool at_T = t >= q->T;
                // the stop rule of kdss_solve: after every `every` iterations
                // (never at t = 0, and once per check point)
                const bool check = o.eps_stop > 0.0 && t > 0 && t % every == 0 && t != q->checked_at;
                q->checked_at = t;
                bool done = false;
                kdss_status qs = KDSS_OK;
                std::string qm;
                if (at_T || check) {
                    int herr = 0;
                    to_host(wctx, &herr, q->st->err.p, 1);
                    if (herr) {
                        qs = KDSS_ERR_CUDA;
                        qm = "FW iteration: water-filling invariant failed on the device";
                        done = true;
                    } else {
                        kdss_result r;
                        memset(&r, 0, sizeof r);
                        try {
                            // in place: the max of r for the bound (zero delta)
                            if (inplace) fw_enqueue_step_range(wctx, *q->st, 0, q->sct->s.n, true);
                            extract_prefix(wctx, q->sct->s, *q->st, &r);
                        } catch (const Error &e) {
                            qs = e.code;
                            qm = e.msg;
                            done = true;
                        }
                        if (qs == KDSS_OK && (at_T || r.gap <= o.eps_stop)) {
                            r.T = q->T;
                            r.status = KDSS_OK;
                            q->res = r;
                            done = true;
                        } else {
                            free(r.ids);
                        }
                    }
                }
                if (!done) { keep.push_back(q); continue; }
                q->st.reset();
                q->sct.reset();  // released on the build stream; this stream is idle
                std::lock_guard<std::mutex> lk(mu);
                resident -= q->bytes;
                finish(q, qs, qm);
                cv_build.notify_all();
                dirty = true;
            }
            active.swap(keep);
            std::lock_guard<std::mutex> lk(mu);
            active_count = (int)active.size();
        } catch (const Error &e) {
            // a device error ends every active query
            drop_exec();
            dirty = true;
            std::lock_guard<std::mutex> lk(mu);
            for (Query *q : active) {
                q->st.reset();
                q->sct.reset();
                resident -= q->bytes;
                finish(q, e.code, e.msg);
            }
            active.clear();
            active_count = 0;
            cv_build.notify_all();
        }
    }
    drop_exec();
    for (Query *q : active) {
        q->st.reset();
        q->sct.reset();
    }
}

namespace {

kdss_status fail_status(const Error &e) {
    set_last_error(e.msg);
    return e.code;
}

}  // namespace

extern "C" {

kdss_status kdss_server_create(const kdss_server_opts *o, kdss_server **out) {
    try {
        if (!o || !out) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
        *out = nullptr;
        if (o->precision != KDSS_INT64 && o->precision != KDSS_FP64 && o->precision != KDSS_FP32K)
            fail(KDSS_ERR_INVALID_ARG, "unknown precision");
        if (o->order != KDSS_ORDER_PEEL && o->order != KDSS_ORDER_CORE)
            fail(KDSS_ERR_INVALID_ARG, "unknown vertex order");
        if (o->check_every < 1) fail(KDSS_ERR_INVALID_ARG, "check_every must be >= 1");
        if ((o->flags & KDSS_FLAG_ASYNC) && o->precision == KDSS_FP32K)
            fail(KDSS_ERR_INVALID_ARG, "in-place iterations need the integer rule");
        if (o->max_active < 0 || o->hbm_budget < 0 || o->eps_stop < 0.0)
            fail(KDSS_ERR_INVALID_ARG, "negative max_active, hbm_budget or eps_stop");
        std::unique_ptr<kdss_server> s(new kdss_server());
        s->o = *o;
        if (s->o.max_active == 0) s->o.max_active = 64;
        KDSS_CUDA(cudaGetDevice(&s->device));
        if (s->o.hbm_budget == 0) {
            size_t fr = 0, tot = 0;
            KDSS_CUDA(cudaMemGetInfo(&fr, &tot));
            s->o.hbm_budget = (int64_t)(0.8 * (double)fr);
        }
        KDSS_CUDA(cudaStreamCreateWithFlags(&s->bstream, cudaStreamNonBlocking));
        KDSS_CUDA(cudaStreamCreateWithFlags(&s->wstream, cudaStreamNonBlocking));
        kdss_opts bo{};
        bo.stream = s->bstream;
        s->bctx = make_ctx(&bo);
        kdss_opts wo{};
        wo.stream = s->wstream;
        s->wctx = make_ctx(&wo);
        s->builder = std::thread([p = s.get()] { p->build_loop(); });
        s->iterator = std::thread([p = s.get()] { p->iterate_loop(); });
        *out = s.release();
    } catch (const Error &e) {
        return fail_status(e);
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return KDSS_ERR_CUDA;
    }
    set_last_error("");
    return KDSS_OK;
}

kdss_status kdss_server_submit(kdss_server *s, const kdss_query *q, int64_t *ticket) {
    try {
        if (!s || !q || !ticket) fail(KDSS_ERR_INVALID_ARG, "NULL argument");
        const kdss_graph_desc &g = q->graph;
        if (q->k < 2 || q->k > 255) fail(KDSS_ERR_INVALID_ARG, "k must be in [2, 255]");
        if (q->T < 0) fail(KDSS_ERR_INVALID_ARG, "T must be >= 0");
        if (g.n < 0 || g.n >= (int64_t)INT32_MAX) fail(KDSS_ERR_INVALID_ARG, "n must be in [0, 2^31 - 1)");
        if (g.m < 0 || g.m > ((int64_t)1 << 30)) fail(KDSS_ERR_INVALID_ARG, "m must be in [0, 2^30]");
        if (g.m > 0 && (!g.src || !g.dst)) fail(KDSS_ERR_INVALID_ARG, "edge arrays are NULL");
        if (g.m > 0 && g.on_device) {
            check_device_array(g.src, (size_t)g.m * sizeof(int32_t), "src", s->bctx.device);
            check_device_array(g.dst, (size_t)g.m * sizeof(int32_t), "dst", s->bctx.device);
        }
        std::unique_ptr<Query> x(new Query());
        x->k = q->k;
        x->T = q->T;
        x->n = g.n;
        x->m = g.m;
        if (g.m > 0 && g.on_device) {
            x->dsrc = DBuf<int32_t>(s->bctx, (size_t)g.m);
            x->ddst = DBuf<int32_t>(s->bctx, (size_t)g.m);
            KDSS_CUDA(cudaMemcpyAsync(x->dsrc.p, g.src, (size_t)g.m * 4, cudaMemcpyDeviceToDevice,
                                      s->bctx.stream));
            KDSS_CUDA(cudaMemcpyAsync(x->ddst.p, g.dst, (size_t)g.m * 4, cudaMemcpyDeviceToDevice,
                                      s->bctx.stream));
            sync(s->bctx);
        } else if (g.m > 0) {
            x->hsrc.assign(g.src, g.src + g.m);
            x->hdst.assign(g.dst, g.dst + g.m);
        }
        x->t_submit = Clock::now();
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) fail(KDSS_ERR_CANCELLED, "the server is shutting down");
        x->ticket = s->next_ticket++;
        *ticket = x->ticket;
        s->pending.push_back(x.get());
        s->table[x->ticket] = std::move(x);
        ++s->submitted;
        s->cv_build.notify_all();
    } catch (const Error &e) {
        return fail_status(e);
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return KDSS_ERR_OOM;
    }
    set_last_error("");
    return KDSS_OK;
}

kdss_status kdss_server_wait(kdss_server *s, int64_t ticket, int32_t timeout_ms, kdss_result *out,
                             kdss_query_timing *timing) {
    if (!s) {
        set_last_error("NULL server");
        return KDSS_ERR_INVALID_ARG;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) {
        set_last_error("unknown ticket");
        return KDSS_ERR_INVALID_ARG;
    }
    Query *q = it->second.get();
    auto ready = [&] { return q->state == QState::Done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        set_last_error("the query has not finished");
        return KDSS_ERR_TIMEOUT;
    }
    if (out) {
        *out = q->res;
        out->status = q->status;
        q->res.ids = nullptr;
    }
    if (timing) {
        memset(timing, 0, sizeof *timing);
        const bool built = q->t_built.time_since_epoch().count() != 0;
        const bool iterated = q->t_first.time_since_epoch().count() != 0;
        if (q->t_build0.time_since_epoch().count() != 0)
            timing->queue_ms = ms_between(q->t_submit, q->t_build0);
        if (built) timing->build_ms = ms_between(q->t_build0, q->t_built);
        if (iterated) {
            timing->wait_ms = ms_between(q->t_built, q->t_first);
            timing->iterate_ms = ms_between(q->t_first, q->t_done);
        }
        timing->latency_ms = ms_between(q->t_submit, q->t_done);
        timing->iterations = q->res.t_used;
        timing->peak_batch = q->peak_batch;
        timing->resident_bytes = q->bytes;
    }
    const kdss_status st = q->status;
    set_last_error(q->msg);
    free(q->res.ids);
    s->table.erase(it);
    return st;
}

kdss_status kdss_server_get_stats(kdss_server *s, kdss_server_stats *out) {
    if (!s || !out) {
        set_last_error("NULL argument");
        return KDSS_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->pending = (int64_t)s->pending.size();
    out->active = s->active_count;
    out->resident_bytes = s->resident;
    out->peak_resident_bytes = s->peak_resident;
    out->hbm_budget = s->o.hbm_budget;
    out->replays = s->replays;
    out->captures = s->captures;
    out->peak_active = s->peak_active;
    set_last_error("");
    return KDSS_OK;
}

void kdss_server_destroy(kdss_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Query *q : s->pending) s->finish(q, KDSS_ERR_CANCELLED, "the server was destroyed");
        s->pending.clear();
    }
    s->cv_build.notify_all();
    s->cv_iter.notify_all();
    if (s->builder.joinable()) s->builder.join();
    if (s->iterator.joinable()) s->iterator.join();
    cudaStreamSynchronize(s->wstream);
    cudaStreamSynchronize(s->bstream);
    for (auto &kv : s->table) {
        kv.second->st.reset();
        kv.second->sct.reset();
        kv.second->dsrc.reset();
        kv.second->ddst.reset();
        free(kv.second->res.ids);
    }
    s->table.clear();
    cudaStreamSynchronize(s->bstream);
    cudaStreamDestroy(s->bstream);
    cudaStreamDestroy(s->wstream);
    delete s;
}

}  // extern "C"
