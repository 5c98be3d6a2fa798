/*
 * kdss.h -- C ABI of the GB300 PSCTL solver (k-clique densest subgraph
 * search by Frank-Wolfe over the succinct clique tree, arxiv 2403.05775).
 *
 * Pipeline (the paper's three steps, Fig. 1): build the SCT index of the
 * k-cliques (Sec. 2), run Frank-Wolfe iterations of PBUpdate over its pairs
 * (Alg. 2-3), sort the nodes by r and return the densest prefix (the final
 * step of Alg. 2).  Every step runs in CUDA kernels on one GPU; this header is the
 * only boundary.  No C++ or torch types cross it.
 *
 * Conventions
 *  - Status: every entry point returns kdss_status (0 = OK, < 0 = error) and
 *    never throws.  kdss_last_error() gives a thread-local message for the
 *    last failing call of the calling thread.
 *  - Ownership: kdss_sct, kdss_state and the ids array of kdss_result are
 *    owned by the library and released with the matching _free call.  Input
 *    arrays are borrowed for the duration of the call only.
 *  - Streams: all device work of a call is ordered on opts->stream (a
 *    cudaStream_t; NULL = the legacy default stream).  Calls return after
 *    that stream has finished the call's work, so host results are final.
 *  - Memory: device memory comes from opts->alloc / opts->free when set
 *    (e.g. a framework's caching allocator), otherwise from
 *    cudaMallocAsync / cudaFreeAsync on the stream.  A handle remembers the
 *    allocator it was created with and frees through it.
 *  - Threads: calls on distinct handles may run concurrently on distinct
 *    streams; a handle must not be used by two calls at once.
 *  - Node ids are int32 in [0, n); n < 2^31 - 1.
 */
#ifndef KDSS_H
#define KDSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t kdss_status;
#define KDSS_OK 0
#define KDSS_ERR_INVALID_ARG (-1)   /* bad k, T, size, NULL pointer, option */
#define KDSS_ERR_BAD_GRAPH (-2)     /* an edge endpoint outside [0, n) */
#define KDSS_ERR_OOM (-3)           /* device allocation failed */
#define KDSS_ERR_OVERFLOW (-4)      /* a count leaves its exact range (128 bits; r: see kdss_fw_iterate) */
#define KDSS_ERR_TIMEOUT (-5)       /* a bounded device wait expired */
#define KDSS_ERR_CUDA (-6)          /* a CUDA runtime call failed */
#define KDSS_ERR_CANCELLED (-7)     /* a batch query was cancelled */
#define KDSS_ERR_UNSUPPORTED (-8)   /* e.g. a pair longer than the kernels take */

/* Representation of the per-node ranking r (Table 2: r(u), the weight a node
 * collected).  KDSS_INT64: exact uint64 cumulative r (rule I).  KDSS_FP64: the
 * same integers held in double (exact below 2^53).  KDSS_FP32K: normalised
 * r/t in float with compensated (error-free) scatter sums, continuous rule. */
#define KDSS_INT64 0
#define KDSS_FP64 1
#define KDSS_FP32K 2

/* PBUpdate rule (kdss_opts.rule).  INTEGER: Alg. 3 as written (whole units,
 * the remainder to the lowest ids of the last plateau, Sec. 3.2); its r is
 * held in KDSS_INT64 or KDSS_FP64.  CONTINUOUS: the same water-filling with
 * a real water level and no floor or remainder (what Alg. 3's unit-by-unit
 * filling tends to as the units shrink); it runs in KDSS_FP32K.  DEFAULT: the
 * rule of the precision.  A rule its precision does not hold is
 * KDSS_ERR_UNSUPPORTED. */
#define KDSS_RULE_DEFAULT 0
#define KDSS_RULE_INTEGER 1
#define KDSS_RULE_CONTINUOUS 2

/* Vertex order of the SCT build.  PEEL: key (peel round, id), a degeneracy
 * order (every vertex has at most core(v) <= delta later neighbours).  CORE:
 * key (core number, id); reproduces the paper's Example 2.2 on its graph G1
 * but bounds the out-degree only by the maximum degree. */
#define KDSS_ORDER_PEEL 0
#define KDSS_ORDER_CORE 1

/* flags */
#define KDSS_FLAG_PROFILE 1u        /* time the FW kernels of every 8th iteration with CUDA events */
#define KDSS_FLAG_KEEP_GRAPH 2u     /* keep the CSR, cores and order in the SCT handle */
#define KDSS_FLAG_ASYNC 4u          /* kdss_fw_iterate: pairs update r in place (see there) */
/* Failure injection for tests of the bounded device waits: the peeling
 * kernel's grid barriers wait for one block more than the grid holds, with a
 * 1 ms limit, so every block gives up at its first barrier, the kernel returns
 * and the build fails with KDSS_ERR_TIMEOUT.  Nothing else is affected. */
#define KDSS_FLAG_TEST_BARRIER_TIMEOUT 8u
/* Integer-rule first step on the root-shared form of the SCT (each pair as
 * 16-bit indices into its root's out-neighbourhood, the neighbourhood's r
 * gathered once per tile) whatever the SCT's size; by default it is used only
 * when the SCT's node stream exceeds 96 MiB (beyond L2). */
#define KDSS_FLAG_ROOTED 16u
/* Iterations as launches per iteration (CUDA graphs of the PBUpdate kernels
 * and the step) even where the resident launch applies.  By default (the
 * integer rule and the FP32 continuous rule alike), when every pair of the
 * SCT has at most 32 nodes and the pairs fit
 * the blocks' shared memory (one block per SM, 12 bytes per pair node: about
 * 18,000 pair nodes per SM), kdss_fw_iterate runs all T iterations in one
 * cooperative launch that keeps the pair stream in shared memory and ends
 * each iteration on a bounded grid barrier.  Both forms give the same r bit
 * for bit in the integer rule (the FP32 rule rounds its sums in another
 * order); with KDSS_FLAG_PROFILE the resident launch is timed as a whole and
 * kdss_timing counts it as T PBUpdate passes with the step inside. */
#define KDSS_FLAG_PER_ITERATION 32u

typedef void *(*kdss_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*kdss_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

typedef struct kdss_opts {
    int32_t precision;      /* KDSS_INT64 | KDSS_FP64 | KDSS_FP32K */
    int32_t order;          /* KDSS_ORDER_PEEL | KDSS_ORDER_CORE */
    uint32_t flags;         /* KDSS_FLAG_* */
    int32_t check_every;    /* solve calls: evaluate the stop rule every j iterations (0 = never) */
    double eps_stop;        /* solve calls: stop once 1 - rho'_max / max r-hat <= eps_stop */
    void *stream;           /* cudaStream_t; NULL = legacy default stream */
    kdss_alloc_fn alloc;    /* optional device allocator (NULL: cudaMallocAsync) */
    kdss_free_fn free;      /* must be set together with alloc */
    void *alloc_ctx;        /* passed back to alloc / free */
    int32_t chunk;          /* integer-rule iterations on the work-queue kernels: tiles of 32
                               pairs per work item (kdss_solve_batch: 0 = autotuned;
                               kdss_fw_iterate / kdss_solve: 0 = the per-class kernels) */
    int32_t threads_per_path; /* lanes per pair of 33..256 nodes in the work-queue kernels:
                               8 or 32 (0 = autotuned in batches, 32 otherwise) */
    int32_t rule;           /* KDSS_RULE_*: 0 = the precision's rule; INTEGER with KDSS_INT64 or
                               KDSS_FP64, CONTINUOUS with KDSS_FP32K (else UNSUPPORTED) */
} kdss_opts;

/* An undirected graph as a raw edge list.  Duplicates, both orientations and
 * self-loops are allowed; the build drops self-loops and duplicates (Sec. 2's
 * simple graph G(V, E)).  src/dst are host pointers, or device pointers when
 * on_device != 0.  Device edge arrays must be device (or managed) memory of
 * the device the call runs on at their first and last entries
 * (cudaPointerGetAttributes); otherwise every call taking the descriptor
 * returns INVALID_ARG before any launch (a batch marks that query alone). */
typedef struct kdss_graph_desc {
    int64_t n;
    int64_t m;
    const int32_t *src;
    const int32_t *dst;
    int32_t on_device;
} kdss_graph_desc;

typedef struct kdss_sct kdss_sct;       /* opaque: device-resident SCT of one (G, k) */
typedef struct kdss_state kdss_state;   /* opaque: device-resident FW state (t, r) */

typedef struct kdss_sct_stats {
    int64_t n;              /* nodes */
    int64_t m;              /* undirected edges of the simple graph */
    int64_t eta_k;          /* |P_k| pairs (Lemma 2.5) */
    int64_t L_k;            /* sum over pairs of |V(P)| */
    uint64_t c_k_lo;        /* |C_k(V)| = sum of n_C (Lemma 2.6), low 64 bits */
    uint64_t c_k_hi;        /* high 64 bits */
    int32_t k;
    int32_t degeneracy;     /* delta = max core number */
    int32_t max_out_degree; /* of the oriented graph used by the build */
    int32_t max_pair_len;   /* max |V(P)| */
    int64_t device_bytes;   /* device memory held by the handle */
    int64_t pairs_per_class[8]; /* pairs per length class of the FW kernels
                                   (|V(P)| <= 8, 16, 32, 256, 1024) */
} kdss_sct_stats;

typedef struct kdss_result {
    int64_t istar;          /* size of the returned prefix V_{i*} */
    int32_t *ids;           /* host array of the istar node ids, ascending (library-owned) */
    uint64_t count_lo;      /* |C_k(V_{i*})| exact, low 64 bits */
    uint64_t count_hi;      /* high 64 bits */
    double density;         /* rho_k(V_{i*}) = count / istar */
    double upper_bound;     /* max_u r(u)/t (FP64) */
    double rho_prime;       /* max_i rho'(V_i) of the sorted prefixes (Thm 3.6) */
    double gap;             /* 1 - rho_prime / upper_bound (>= 0 by Thms 3.5-3.6) */
    int32_t T;              /* iterations requested */
    int32_t t_used;         /* iterations run */
    kdss_status status;     /* per-query status in batch calls */
    int32_t reserved;
} kdss_result;

typedef struct kdss_timing {
    double fw_kernel_ms;    /* summed event time of the timed PBUpdate passes */
    double step_kernel_ms;  /* summed event time of the timed step kernels */
    int64_t fw_launches;    /* PBUpdate passes timed (every 8th iteration; every iteration of
                               a resident launch, whose time includes its steps) */
    int64_t step_launches;
} kdss_timing;

/*
 * kdss_build_sct -- steps A1-A3: simple graph in CSR, core numbers and vertex
 * order, and the SCT restricted to P_k (Sec. 2, Lemmas 2.4-2.6): pairs
 * (V_h, V_p) with |V_h| <= k <= |V(P)| whose k-cliques partition C_k(V).
 *   g    : the input graph (host or device edge list).
 *   k    : clique size, 2 <= k <= 255.
 *   opts : stream, allocator, order.
 *   out  : receives the new handle (NULL on error).
 * Clique counts are exact: n_C = C(p, k - h) of every pair and c_k in
 * 128 bits (c_k_lo / c_k_hi of kdss_sct_stats).  The integer-rule
 * iterations need t * c_k < 2^63 (KDSS_INT64) or 2^53 (KDSS_FP64); the FP32
 * rule takes every count below 2^128 (rounded to float).
 * Errors: INVALID_ARG (k, n, m, NULL), BAD_GRAPH (id outside [0, n)),
 *   OVERFLOW (a count needs more than 128 bits), UNSUPPORTED (a pair
 *   longer than 1024 nodes), OOM, CUDA.
 */
kdss_status kdss_build_sct(const kdss_graph_desc *g, int32_t k, const kdss_opts *opts,
                           kdss_sct **out);

/* Sizes of P_k measured by kdss_sct_count. */
typedef struct kdss_sct_count_stats {
    int64_t eta_k;          /* |P_k| over the roots walked to the end */
    int64_t L_k;            /* sum of |V(P)| over those pairs */
    uint64_t c_k_lo;        /* sum of n_C over those pairs, low 64 bits */
    uint64_t c_k_hi;        /* high 64 bits */
    int64_t pairs_per_class[8]; /* |V(P)| <= 8, 16, 32, 256, 1024, longer (6 used) */
    int64_t roots_total;    /* n */
    int64_t roots_done;     /* roots whose recursion was walked to the end */
    int64_t roots_cut;      /* roots the time budget interrupted (not in the counts) */
    int64_t cut_pairs;      /* pairs the interrupted roots had emitted */
    int64_t cut_nodes;      /* their node entries */
    int64_t m;              /* undirected edges of the simple graph */
    int32_t complete;       /* 1: every root walked, the counts are exact */
    int32_t max_pair_len;   /* longest pair seen */
    int32_t degeneracy;
    int32_t max_out_degree;
    int32_t count_bits;     /* bit length of the largest n_C seen (129: beyond 128 bits) */
    int32_t reserved;
    double seconds;         /* device time of the counting kernel */
} kdss_sct_count_stats;

/*
 * kdss_sct_count -- the sizes of P_k (eta_k, L_k, c_k, pairs per length class;
 * Sec. 2, Lemmas 2.4-2.6) without storing a pair, for SCTs far beyond the
 * device (Thm 3.7: the SCT takes O(eta) space).  Steps A1-A2 run as in
 * kdss_build_sct; then one warp walks each root's recursion to the end, the
 * roots taken in the order i -> (i * P) mod n (P a fixed prime not dividing
 * n), until every root is done or budget_s seconds of device time have
 * passed (budget_s = 0: no limit).  The counts cover the roots walked to the
 * end; when `complete` is 0 those roots are a pseudo-random sample of all
 * roots, so (counts) * roots_total / roots_done estimates the whole SCT.
 * Out-degrees up to 4095 are taken (pairs of up to 4096 nodes are counted
 * in the last class even though the FW kernels stop at 1024).
 * Errors: INVALID_ARG, BAD_GRAPH, UNSUPPORTED (out-degree above 4095), OOM,
 *   CUDA.
 */
kdss_status kdss_sct_count(const kdss_graph_desc *g, int32_t k, double budget_s,
                           const kdss_opts *opts, kdss_sct_count_stats *out);

/*
 * kdss_sct_from_pairs -- make an SCT handle from caller-given pairs, so the
 * FW and extraction steps can run on an SCT built elsewhere.  Pair q holds
 * nodes[pair_off[q] .. pair_off[q+1]) with its first h[q] entries the hold
 * set V_h and the rest the pivot set V_p (Sec. 2, Lemma 2.4); 0 <= h <= k <=
 * |V(P)| <= 1024 is required.  Arrays are host pointers, or device pointers when
 * on_device != 0; they are copied.  Device arrays must be device (or managed)
 * memory of the current device at their first and last entries
 * (cudaPointerGetAttributes), else INVALID_ARG before any launch.
 * Errors: INVALID_ARG (sizes, h, k, ids outside [0, n)), OVERFLOW, OOM, CUDA.
 */
kdss_status kdss_sct_from_pairs(int64_t n, int32_t k, int64_t npairs, const int64_t *pair_off,
                                const int32_t *nodes, const int32_t *h, int32_t on_device,
                                const kdss_opts *opts, kdss_sct **out);

/* kdss_sct_info -- sizes of the handle (eta_k, L_k, c_k, delta ...). */
kdss_status kdss_sct_info(const kdss_sct *s, kdss_sct_stats *out);

/*
 * kdss_sct_copy_pairs -- copy the pairs to host buffers of eta_k + 1, L_k and
 * eta_k entries.  Layout as stored on the device: pairs grouped by length
 * class, within a pair the nodes ascending by id with bit 31 set on hold
 * (V_h) nodes; h[q] = |V_h|.
 */
kdss_status kdss_sct_copy_pairs(const kdss_sct *s, int64_t *pair_off, int32_t *nodes,
                                int32_t *h);

/*
 * kdss_sct_copy_graph -- copy step A1-A2 outputs to host buffers: CSR offsets
 * (n + 1) and neighbours (2 m), core numbers, peel rounds and the rank of
 * every vertex in the build order (n each).  Any pointer may be NULL.  Only
 * for handles built with KDSS_FLAG_KEEP_GRAPH (INVALID_ARG otherwise).
 */
kdss_status kdss_sct_copy_graph(const kdss_sct *s, int64_t *off, int32_t *adj, int32_t *core,
                                int32_t *round_, int32_t *rank);

/*
 * kdss_build_sct_multi -- a k-agnostic SCT: steps A1-A3 with the pruning of
 * Lemma 2.5 relaxed to |V_h| <= k_max and |V(P)| >= 2, so that the handle
 * holds P_k for every k in [2, k_max] at once (P_k = the pairs with
 * |V_h| <= k <= |V(P)|, Sec. 2).  It is built once per graph and cut to one
 * k by kdss_sct_restrict, or iterated at any k where it stands by
 * kdss_fw_iterate_at (kdss_fw_iterate without a k refuses it).
 * kdss_sct_info reports every kept pair (eta, L), k = k_max and
 * c_k = c_{k_max}.
 * Errors: as kdss_build_sct.
 */
kdss_status kdss_build_sct_multi(const kdss_graph_desc *g, int32_t k_max, const kdss_opts *opts,
                                 kdss_sct **out);

/*
 * kdss_sct_restrict -- P_k of a k-agnostic SCT (2 <= k <= its k_max): the
 * pairs with |V_h| <= k <= |V(P)|, in the stored order, with the binomial
 * table and c_k of k -- the same pairs kdss_build_sct(g, k) emits.
 * *out is a new, ordinary SCT handle (free it with kdss_sct_free).
 * Errors: INVALID_ARG (not k-agnostic, k out of range), OVERFLOW, OOM, CUDA.
 */
kdss_status kdss_sct_restrict(const kdss_sct *multi, int32_t k, const kdss_opts *opts,
                              kdss_sct **out);

/*
 * kdss_fw_iterate -- step A4-A5: T Frank-Wolfe iterations of Alg. 2 with the
 * PBUpdate rule of Alg. 3 over every pair, all pairs of iteration t reading
 * r_{t-1} (synchronous form); the remainder units of Alg. 3 (fewer than the
 * plateau's size, placed at random in the paper) go to the lowest node ids;
 * r_0 = 0.  *state is created when NULL (precision from
 * opts), otherwise continued from its iteration count t.
 *   s     : SCT handle.
 *   state : in/out FW state.
 *   T     : iterations to run, T >= 0.
 * With KDSS_FLAG_ASYNC (integer rule, KDSS_INT64 / KDSS_FP64 only) the pairs
 * add their allocations straight into r while others read it, the way Alg. 2
 * as printed updates r in place pair after pair: a pair reads r as it stands
 * when it loads it (updates made earlier in the same iteration may or may
 * not be visible), so the result depends on the schedule and is not
 * reproducible; each pair still hands out exactly its n_C units within its
 * caps, so sum_u r_t(u) = t c_k and r_t / t stays feasible.
 * Errors: INVALID_ARG, OVERFLOW (r would leave the exact range), OOM,
 *   UNSUPPORTED (KDSS_FLAG_ASYNC with KDSS_FP32K), CUDA.
 */
kdss_status kdss_fw_iterate(kdss_sct *s, kdss_state **state, int32_t T, const kdss_opts *opts);

/*
 * kdss_fw_iterate_at -- kdss_fw_iterate at a chosen k.  On a k-agnostic SCT
 * (kdss_build_sct_multi, 2 <= k <= its k_max) the iterations run over P_k
 * where it stands: by Lemma 2.5 P_k is the set of pairs with
 * |V_h| <= k <= |V(P)|, and the kernels skip every other pair, so one handle
 * serves every k without a copy (kdss_sct_restrict makes the copy instead).
 * On a k-pruned SCT k must be its own k.  A new state records k and c_k of
 * P_k; a continued state must have been created with the same k.
 * kdss_extract then extracts at the state's k.
 * Errors: as kdss_fw_iterate; INVALID_ARG (k outside the SCT's range, a
 *   state of another k).
 */
kdss_status kdss_fw_iterate_at(kdss_sct *s, int32_t k, kdss_state **state, int32_t T,
                               const kdss_opts *opts);

/*
 * kdss_sct_share_prefixes -- the prefix-shared form of an SCT's pairs (Sec. 2,
 * Lemmas 2.4-2.5: the pairs of one recursion repeat its hold and pivot
 * nodes).  Within each length class the pairs are put in lexicographic order
 * of their node lists (ids ascending, V_h and V_p marked), and each pair keeps
 * only the nodes after the prefix it shares with the pair before it; every
 * block of 32 pairs starts with a pair kept whole.  The kept nodes are the
 * nodes of the prefix tree of the pairs, so equal prefixes are stored once.
 *   in          : a k-pruned or k-agnostic SCT handle (flat pairs); it stays
 *                 valid and owned by the caller.
 *   chunk_pairs : pairs decoded at a time when iterating or extracting
 *                 (rounded to whole blocks; 0 = 2^22).
 *   out         : a new handle (free it with kdss_sct_free) holding the
 *                 shared form, the counts and the binomial tables, and no
 *                 graph.
 * The new handle iterates with kdss_fw_iterate / kdss_fw_iterate_at
 * (synchronous rule, any precision; r_T equal bit for bit to the flat
 * handle's in the integer rule) and extracts with kdss_extract: each
 * iteration decodes one chunk at a time into the flat layout on the device
 * and runs the same PBUpdate kernels, so the flat pairs exist one chunk at a
 * time.  kdss_sct_info reports the same eta_k, L_k and c_k, and device_bytes
 * of the shared form; kdss_sct_copy_pairs returns the pairs in the shared
 * order.  KDSS_FLAG_ASYNC, work-queue chunks, kdss_sct_restrict, the explicit
 * clique list and kdss_fw_iterate_noalloc need the flat handle (INVALID_ARG or
 * UNSUPPORTED).
 * Errors: INVALID_ARG (NULL, chunk_pairs < 0, a shared input), UNSUPPORTED
 *   (2^31 pairs or more), OOM, CUDA.
 */
kdss_status kdss_sct_share_prefixes(const kdss_sct *in, int64_t chunk_pairs, const kdss_opts *opts,
                                    kdss_sct **out);

/*
 * kdss_sct_shared_words -- node words kept by a prefix-shared SCT (against
 * L_k of the flat pairs) and the chunks an iteration decodes.  Either output
 * may be NULL.  Errors: INVALID_ARG (NULL handle, not prefix-shared).
 */
kdss_status kdss_sct_shared_words(const kdss_sct *s, int64_t *words, int64_t *chunks);

/*
 * kdss_fw_cliques -- T iterations of Alg. 1 (the Frank-Wolfe step over the
 * explicit k-clique list): every k-clique gives its unit to its member of
 * least (r, id), all cliques of iteration t reading r_{t-1} (synchronous
 * form, as kdss_fw_iterate).  The list is the expansion of the SCT (each pair
 * (V_h, V_p) holds V_h + S for the (k - |V_h|)-subsets S of V_p, Lemmas
 * 2.4-2.5), built on the device on first use and kept in the handle.  The
 * state is an ordinary KDSS_INT64 state, so kdss_extract applies; r_t / t is
 * feasible for CP(G) and max r / t bounds rho_k(V*) from above (Lemma 2.3).
 *   s, state, T : as for kdss_fw_iterate (opts->precision must be KDSS_INT64).
 * Errors: INVALID_ARG, UNSUPPORTED (precision), OOM (the list would take
 *   more than half of the free device memory; the message gives its size),
 *   OVERFLOW, CUDA.
 */
kdss_status kdss_fw_cliques(kdss_sct *s, kdss_state **state, int32_t T, const kdss_opts *opts);

/*
 * kdss_sct_copy_cliques -- the explicit k-clique list of kdss_fw_cliques
 * (expanded on first use): min(capacity, c_k) rows of k node ids are copied
 * to the host buffer `cliques`; *count receives c_k.  Rows come grouped by
 * pair, hold ids first.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
kdss_status kdss_sct_copy_cliques(kdss_sct *s, int32_t *cliques, int64_t capacity, int64_t *count);

/* Counters of a kdss_cpsample run. */
typedef struct kdss_cpsample_stats {
    uint64_t paths_total;     /* k-color paths (strictly increasing colours) */
    int64_t samples;          /* paths drawn (t) */
    int64_t samples_clique;   /* drawn paths that are k-cliques */
    int64_t cliques;          /* distinct k-cliques among them (the sample set) */
    int32_t colors;           /* colours of the greedy colouring */
    int32_t reserved;
} kdss_cpsample_stats;

/*
 * kdss_cpsample -- CPSample (Sec. 5, Alg. 4): t uniform k-color paths (the
 * CCPATH sampler: a greedy colouring, then paths whose colours increase; a
 * clique's members sorted by colour form exactly one such path, so uniform
 * paths give uniform cliques), the set of k-cliques among them, T iterations
 * of Alg. 1 over that set (synchronous form), and the prefix of the nodes
 * sorted by r with the largest |C_k(V_i) & set| / i.  No SCT is built.
 * Readings: the colouring is greedy by decreasing rank of the build order
 * (opts->order), each vertex taking the smallest colour its coloured
 * neighbours lack; sample j takes word j of SplitMix64 seeded with `seed`,
 * x, and the path of rank floor((x >> 11) * #paths / 2^53) in the order
 * (start id, then adjacency order); repeated cliques count once.
 *   g     : input graph, as for kdss_build_sct.
 *   k     : 2..16.   t : samples, 0..2^31.   T : Alg. 1 iterations >= 0.
 *   out   : istar, ids (library-owned, kdss_result_free), count_lo =
 *           |C_k(V_i*) & set|, density = count_lo / istar (the sampled
 *           density), upper_bound = max r / T.
 *   stats : may be NULL.
 * Errors: INVALID_ARG, BAD_GRAPH, OVERFLOW (path counts beyond 63 bits),
 *   UNSUPPORTED (a vertex with more than 4095 higher-ranked neighbours), OOM,
 *   CUDA.
 */
kdss_status kdss_cpsample(const kdss_graph_desc *g, int32_t k, int64_t t, int32_t T, uint64_t seed,
                          const kdss_opts *opts, kdss_result *out, kdss_cpsample_stats *stats);

/*
 * kdss_state_copy_r -- copy r to a host buffer of n entries: uint64 for
 * KDSS_INT64 (cumulative r_t), double for KDSS_FP64 (cumulative r_t), float
 * for KDSS_FP32K (normalised r_t / t).  *t_out receives t (may be NULL).
 */
kdss_status kdss_state_copy_r(const kdss_state *st, void *r_host, int32_t *t_out);

/* kdss_state_timing -- event times of the FW kernels (KDSS_FLAG_PROFILE). */
kdss_status kdss_state_timing(const kdss_state *st, kdss_timing *out);

/*
 * kdss_extract -- step A6 (the final step of Alg. 2): sort the nodes by r
 * non-increasing (ties by ascending id), count the k-cliques of every prefix
 * V_i exactly from the pairs (Lemmas 2.5-2.6), and return the prefix of
 * largest rho_k(V_i) = |C_k(V_i)| / i (largest i on ties), with the bound
 * max_u r(u)/t and max_i rho'(V_i) (Thms 3.5-3.6).
 * The k is the state's (kdss_fw_iterate_at on a k-agnostic SCT).
 * out->ids is a library-owned host array (kdss_result_free).
 * Errors: INVALID_ARG, OVERFLOW, OOM, CUDA.
 */
kdss_status kdss_extract(const kdss_sct *s, const kdss_state *st, const kdss_opts *opts,
                         kdss_result *out);

/* kdss_solve -- build, iterations and extraction in one call.  Runs T
 * iterations; with opts->check_every = j > 0 and opts->eps_stop = eps > 0 it
 * extracts after every j iterations and stops early once the certificate gap
 * 1 - rho'_max / max r-hat (Thms 3.5-3.6) is <= eps (out->t_used holds the
 * iterations run). */
kdss_status kdss_solve(const kdss_graph_desc *g, int32_t k, int32_t T, const kdss_opts *opts,
                       kdss_result *out);

/*
 * kdss_solve_streamed -- kdss_solve (build, T iterations, extraction) for
 * graphs whose SCT does not fit the device.  The roots of the build order
 * are split into nchunks equal ranges; every iteration rebuilds the pairs of
 * one range at a time (step A3 restricted to those roots), adds their
 * PBUpdate allocations (Alg. 3) into the shared delta and frees them, then
 * takes the step; the extraction visits the ranges the same way.  All pairs
 * of an iteration still read r_{t-1}, so the result equals kdss_solve's:
 * bit for bit for KDSS_INT64 and KDSS_FP64 (integer sums), the same rule for
 * KDSS_FP32K.  Device memory holds the graph, the state and one range's
 * pairs; each iteration costs nchunks SCT builds.
 *   nchunks : number of root ranges, >= 1 (1 = one build per iteration).
 *   opts    : precision, order, stream, allocator (no stop rule, no
 *             KDSS_FLAG_ASYNC).
 * Errors: as kdss_solve; UNSUPPORTED with KDSS_FLAG_ASYNC.
 */
kdss_status kdss_solve_streamed(const kdss_graph_desc *g, int32_t k, int32_t T, int32_t nchunks,
                                const kdss_opts *opts, kdss_result *out);

/* One query of a batch. */
typedef struct kdss_query {
    kdss_graph_desc graph;
    int32_t k;
    int32_t T;
} kdss_query;

/*
 * kdss_solve_batch -- solve nq independent (graph, k, T) queries (the
 * paper solves one graph at a time; batching is this library's addition).
 * Queries with equal (k, T) are joined into one disjoint-union graph (node
 * ids shifted), which goes through one CSR build, one peeling and one SCT
 * build: peeling acts on each connected component separately, so every
 * query gets the order, the SCT and therefore the r it would get alone.
 * All groups then iterate together (one CUDA graph per iteration; a group
 * drops out after its T), and one segmented sort and scan per group extract
 * every query's densest prefix.
 *   q[i]   : the query (graph as in kdss_build_sct, k in [2, 255], T >= 0).
 *   out[i] : caller-owned; receives query i's result and status (ids
 *            allocated by the library, freed with kdss_result_free).
 *   opts   : as for kdss_solve (one precision and order for all queries);
 *            every query runs its T iterations (no early stop).
 * Results equal kdss_solve's per query: bit for bit for KDSS_INT64 and
 * KDSS_FP64; for KDSS_FP32K the same rule in the same precision (its atomic
 * sums round in the order the hardware performs them, run to run, as in
 * kdss_solve).
 * A query that is invalid, has an edge endpoint outside [0, n) or leaves the
 * exact range gets its own error status and a zeroed result; the others are
 * solved.  Returns OK when every query succeeded, else the first failing
 * query's status (its message in kdss_last_error); an error of the whole
 * batch (device memory, CUDA) is every query's status.
 */
kdss_status kdss_solve_batch(const kdss_query *q, int32_t nq, kdss_result *out,
                             const kdss_opts *opts);

/* What the last kdss_solve_batch of the calling thread ran its iterations
 * with: the chunk (tiles of 32 pairs per work item of the work-queue pass;
 * 0 = each group's per-class kernels in turn) and lanes per long pair it used
 * and, when it tuned them, the configurations it timed (one iteration each,
 * after two warm-up iterations; every one of those is an iteration of the
 * run). */
typedef struct kdss_batch_tuning {
    int32_t chunk;
    int32_t threads_per_path;
    int32_t autotuned;      /* 1 when the candidates below were timed */
    int32_t ntried;
    int32_t tried_chunk[8];
    int32_t tried_threads_per_path[8];
    float tried_ms[8];      /* CUDA-event time of the candidate's iteration */
} kdss_batch_tuning;
kdss_status kdss_batch_last_tuning(kdss_batch_tuning *out);

void kdss_sct_free(kdss_sct *s);
void kdss_state_free(kdss_state *st);
void kdss_result_free(kdss_result *r);   /* frees r->ids; the struct is caller-owned */

/* Thread-local message of the calling thread's last error ("" if none). */
const char *kdss_last_error(void);

/* Library version string. */
const char *kdss_version(void);

/* Number of CUDA kernels this library has launched in the process so far
 * (all threads); the difference of two calls counts the launches between. */
int64_t kdss_kernel_launches(void);

/*
 * kdss_fw_iterate_noalloc -- the FW iterations of kdss_fw_iterate (integer
 * rule, KDSS_INT64 semantics) without any device allocation.  The paper has
 * no counterpart: this is an interface for callers that cannot allocate
 * device memory while they iterate -- a process whose GPU memory is reserved
 * up front and handed out by its own arena, a serving loop held to a fixed
 * footprint, code that must not slip an implicitly synchronising cudaMalloc
 * between its kernels.
 *   s      : SCT handle, built beforehand (kdss_build_sct / _from_pairs) on
 *            the current device.
 *   r      : caller-owned device array of n uint64, the cumulative r after
 *            t_done iterations (zeros for t_done = 0); updated in place to r
 *            after t_done + T iterations.  Its first and last elements must
 *            be device (or managed) memory of the current device
 *            (cudaPointerGetAttributes); otherwise INVALID_ARG, before any
 *            launch.
 *   t_done : iterations already in r (only bounds the exact range of r).
 *   T      : iterations to run, T >= 0.
 *   stream : cudaStream_t the work is ordered on.  The call is synchronous:
 *            it reads the device error word back and waits for the stream
 *            before it returns.
 * Scratch: the per-iteration delta and the work lists live in one fixed
 * device array of 16 MiB inside the library, which every GPU that loads the
 * library holds until the process exits.  It fits graphs with
 * 8 * n + 4 * (pairs of at most 32 nodes) + 768 bytes <= 16 MiB (about two
 * million nodes); larger inputs are rejected with KDSS_ERR_INVALID_ARG and a
 * message that states the sizes.  The array keeps the previous call's
 * contents; each call clears what must start at zero.  All calls share it:
 * calls that overlap on the GPU (other streams, other host threads) race and
 * must be serialised by the caller.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and caches it with the
 * device's current context; make that first call before any stream capture.
 * A call in a new context of the device (after cudaDeviceReset) looks the
 * address up again.  No cudaMalloc, cudaFree or
 * allocating library routine is called.
 * Errors: INVALID_ARG (NULL, T < 0, sizes above the scratch, another device),
 *   OVERFLOW, CUDA.
 */
kdss_status kdss_fw_iterate_noalloc(const kdss_sct *s, uint64_t *r, int32_t t_done, int32_t T,
                                    void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KDSS_H */
