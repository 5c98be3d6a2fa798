/*
 * kdss_server.h -- continuous-batching query server on top of kdss.h.
 *
 * The paper solves one (graph, k) at a time; serving many queries is this
 * library's addition.  A server owns two host threads and two CUDA streams on
 * the current device:
 *  - the builder takes submitted queries in arrival order and builds their
 *    SCTs (steps A1-A3, Sec. 2) while the resident footprint (SCTs plus FW
 *    states of admitted queries) is below the HBM budget;
 *  - the iterator runs Frank-Wolfe iterations (Alg. 2-3, the same kernels as
 *    kdss_fw_iterate) for every admitted query together: one CUDA graph per
 *    set of active queries, replayed; a query joins at the next replay after
 *    its build and leaves when it stops.
 * Builds on one stream overlap the iterations of the admitted queries on the
 * other.  A query stops at its T, or earlier once the certificate gap
 * 1 - rho'_max / max r-hat (Thms 3.5-3.6) is <= eps_stop, evaluated after
 * every check_every of its own iterations -- the rule of kdss_solve with the
 * same options, so a query's result does not depend on the other queries it
 * ran with (bit for bit for KDSS_INT64 / KDSS_FP64).  With KDSS_FLAG_ASYNC
 * the queries iterate in place (kdss_fw_iterate's in-place form), which
 * reaches the gap in fewer iterations; results then depend on the schedule.
 * All device memory comes from cudaMallocAsync on the server's streams
 * (allocator callbacks in the options are not used); the caller's stream in
 * the options is not used either.
 */
#ifndef KDSS_SERVER_H
#define KDSS_SERVER_H

#include "kdss.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kdss_server kdss_server;  /* opaque */

typedef struct kdss_server_opts {
    int32_t precision;      /* KDSS_INT64 | KDSS_FP64 | KDSS_FP32K */
    int32_t order;          /* KDSS_ORDER_PEEL | KDSS_ORDER_CORE */
    int32_t check_every;    /* stop-rule period in iterations, >= 1 */
    int32_t max_active;     /* queries iterated together at most (0: 64) */
    double eps_stop;        /* certificate gap to stop at (0: run T iterations) */
    int64_t hbm_budget;     /* bytes of SCTs + states resident at once
                               (0: 80% of the device memory free at creation) */
    uint32_t flags;         /* KDSS_FLAG_ASYNC: in-place iterations (integer rule
                               only; results then depend on the schedule) */
    int32_t reserved;
} kdss_server_opts;

typedef struct kdss_query_timing {
    double queue_ms;        /* submit -> start of its SCT build */
    double build_ms;        /* SCT build (steps A1-A3) */
    double wait_ms;         /* built -> first iteration */
    double iterate_ms;      /* first iteration -> result */
    double latency_ms;      /* submit -> result */
    int32_t iterations;     /* FW iterations run */
    int32_t peak_batch;     /* most queries iterated together while it ran */
    int64_t resident_bytes; /* its SCT + state footprint */
} kdss_query_timing;

typedef struct kdss_server_stats {
    int64_t submitted, completed, failed;
    int64_t pending, active;
    int64_t resident_bytes, peak_resident_bytes, hbm_budget;
    int64_t replays;        /* fused iteration launches (CUDA graph replays) */
    int64_t captures;       /* CUDA graphs captured (one per active set) */
    int32_t peak_active;
    int32_t reserved;
} kdss_server_stats;

/*
 * kdss_server_create -- start a server on the current device.
 * Errors: INVALID_ARG (precision, order, check_every < 1, negative sizes),
 *   CUDA.
 */
kdss_status kdss_server_create(const kdss_server_opts *o, kdss_server **out);

/*
 * kdss_server_submit -- queue one query; returns at once.  The edge list is
 * copied (host arrays into host memory, device arrays into device memory on
 * the builder's stream), so the caller may release it after the call.
 *   ticket : receives the query's id for kdss_server_wait.
 * Errors: INVALID_ARG (k in [2, 255], T >= 0, n, m, NULL arrays), CANCELLED
 *   (the server is shutting down), OOM, CUDA.
 */
kdss_status kdss_server_submit(kdss_server *s, const kdss_query *q, int64_t *ticket);

/*
 * kdss_server_wait -- wait up to timeout_ms (< 0: no limit) for a query's
 * result.  On completion the result (library-allocated ids, freed with
 * kdss_result_free) and its timing are moved to the caller and the ticket is
 * retired; the return value is the query's own status (BAD_GRAPH, OVERFLOW,
 * OOM when its SCT does not fit the budget alone, ...).
 * Errors: INVALID_ARG (unknown ticket), TIMEOUT (not finished yet; the ticket
 *   stays valid).
 */
kdss_status kdss_server_wait(kdss_server *s, int64_t ticket, int32_t timeout_ms, kdss_result *out,
                             kdss_query_timing *timing);

/* kdss_server_get_stats -- counters of the server so far. */
kdss_status kdss_server_get_stats(kdss_server *s, kdss_server_stats *out);

/* kdss_server_destroy -- cancel queued queries, finish nothing more, join
 * the threads and free every resource. */
void kdss_server_destroy(kdss_server *s);

#ifdef __cplusplus
}
#endif
#endif /* KDSS_SERVER_H */
