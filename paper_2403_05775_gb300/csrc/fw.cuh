// fw.cuh -- Frank-Wolfe state and iterations (steps A4-A5).
#pragma once

#include <functional>

#include "sct.cuh"

namespace kdss {

// One SCT of a work-queue iteration (device copy of its arrays' addresses).
struct QGroup {
    const int64_t *pair_off;
    const int32_t *nodes;
    const uint8_t *h;
    const uint64_t *binom;
    const float *binomf;
    int bcols, k;
    int64_t node_off;     // its slice of the shared state
    int64_t short_end;    // pairs [0, short_end) have at most 32 nodes
    int64_t long_begin[2], long_end[2];   // pairs of 33..256 and 257..1024 nodes
};

// A work item of the queue kernels.
struct QItem {
    int32_t g;        // SCT (group) index
    int32_t kind;     // 0: tiles of short pairs; 1: pairs of 33..256 nodes; 2: 257..1024
    int64_t first;    // first tile (kind 0) or first pair (kinds 1, 2)
    int32_t count;    // tiles or pairs
    int32_t pad;
};
// The groups and items of one work-queue PBUpdate pass over several SCTs.
struct QueuePlan {
    DBuf<QGroup> groups;
    DBuf<QItem> items;
    DBuf<unsigned> cursor;
    int nitems = 0;    // items of short pairs (first in `items`)
    int nlong[2] = {0, 0};   // then items of pairs of 33..256 and of 257..1024 nodes
    int chunk = 4;     // tiles of 32 short pairs per item (8 x chunk longer pairs)
    int tpp = 32;      // lanes per pair of 33..256 nodes (8 or 32)
};

struct StateDev {
    int precision = KDSS_INT64;
    int64_t n = 0;
    int t = 0;                       // iterations done
    int k = 0;                       // the k iterated (P_k of the SCT)
    uint64_t ck_lo = 0, ck_hi = 0;   // its c_k
    DBuf<uint64_t> r;                // [n] uint64 or double bits (rule I), cumulative
    DBuf<uint64_t> acc;              // [n] per-iteration delta (same type as r)
    DBuf<float> r32;                 // [n] FP32K: normalised r / t
    DBuf<float> r32c;                // [n] FP32K: Kahan compensation of r32
    DBuf<float> a32;                 // [n] FP32K: per-iteration allocation (hi)
    DBuf<float> a32c;                // [n] FP32K: error terms of the allocation sum
    DBuf<unsigned long long> maxr;   // [1] max r (uint64 / double bits / float bits)
    DBuf<int> err;                   // [1] device error word
    DBuf<int32_t> ovf_list;          // pairs of <= 32 nodes left to the full walk
    DBuf<int> ovf_count;             // their number (reset by the step kernel)
    DBuf<int> dev_t;                 // [0] iterations done (FP32 schedule), [1] scratch
    kdss_timing timing{};
    Ctx ctx;
    int qchunk = 0, qtpp = 32;       // > 0: integer-rule passes on the work-queue kernels
    bool force_rooted = false;       // the root-shared first step whatever the SCT's size
    QueuePlan qplan;                 // their plan, bound like the graphs to one SCT
    bool per_iteration = false;      // no resident launch: per-iteration kernels only
    // resident iterations (all T in one cooperative launch): the second
    // copy of r, the two extra delta vectors, the shares' local indices and
    // distinct nodes, and the largest share, bound like the graphs to one SCT
    const SctDev *res_sct = nullptr;
    int res_state = 0;               // 1: usable for res_sct, -1: not usable
    DBuf<uint64_t> res_r1, res_a1, res_a2;
    DBuf<GridBarrier> res_bar;
    DBuf<uint16_t> res_lidx;         // [nnodes] local index of every pair node in its share
    DBuf<uint16_t> res_loff;         // [npairs] offset of every pair in its share's node list
    DBuf<int32_t> res_uid;           // distinct nodes of every share
    DBuf<int> res_plan;              // [2G] distinct nodes and pair nodes of every share
    int res_ncap = 0, res_pcap = 0, res_ucap = 0;
    size_t res_smem = 0;
    // one FW iteration as CUDA graphs, bound to the SCT they were captured for
    const SctDev *graph_sct = nullptr;
    cudaGraphExec_t g_iter = nullptr, g_pb = nullptr, g_step = nullptr;
    long long nk_pb = 0, nk_step = 0;
    std::vector<cudaEvent_t> events;  // timing events (KDSS_FLAG_PROFILE)
    StateDev() = default;
    StateDev(const StateDev &) = delete;
    StateDev &operator=(const StateDev &) = delete;
    ~StateDev();
    void release_graphs();
};

// Entries of the list of pairs the first-step kernels leave to the slow
// kernels (at most every short pair).
int64_t slow_list_capacity(int64_t short_pairs, int num_sms);
// k < 0: the SCT's own k; otherwise iterate P_k of a k-agnostic SCT.
void fw_init(const Ctx &c, const SctDev &s, int precision, StateDev &st, int k = -1);
void fw_run(const Ctx &c, const SctDev &s, StateDev &st, int T, bool profile);
// in-place (asynchronous) iterations of the integer rule: pairs add into r
void fw_run_async(const Ctx &c, const SctDev &s, StateDev &st, int T);
void fw_enqueue_inplace(const Ctx &c, const SctDev &s, StateDev &st);
// batches: several SCTs over disjoint node ranges of one state
void fw_init_n(const Ctx &c, int64_t n, int64_t short_capacity, int precision, StateDev &st);
// k < 0: the SCT's own k; otherwise P_k of a k-agnostic SCT (the P_k filter).
void fw_enqueue_group(const Ctx &c, const SctDev &s, StateDev &st, int64_t node_off, int k = -1);
void fw_enqueue_step_range(const Ctx &c, StateDev &st, int64_t node_off, int64_t n, bool advance);
long long fw_capture(const Ctx &c, cudaGraphExec_t *exec, const std::function<void(const Ctx &)> &fn);
// Work-queue PBUpdate: one launch over every (SCT, state slice) of `sets`.
// k >= 0: iterate P_k of every set's SCT at that k (the P_k filter).
void queue_plan(const Ctx &c, const std::vector<std::pair<const SctDev *, int64_t>> &sets, int chunk,
                int tpp, QueuePlan &qp, int k = -1);
void queue_enqueue(const Ctx &c, QueuePlan &qp, StateDev &st);
// Extraction (A6) in phases, for pairs that come in pieces.
struct PrefixAcc {
    int64_t n = 0;
    bool wide = false;           // 128-bit prefix counts
    double rmax = 0;             // max_u r(u)/t
    DBuf<int32_t> order, pos;
    DBuf<unsigned long long> hist, fhist;
    DBuf<U128> hist128, fhist128;
};
void prefix_begin(const Ctx &c, int64_t n, const StateDev &st, bool wide, PrefixAcc &a);
void prefix_add(const Ctx &c, const SctDev &s, int k, PrefixAcc &a);
void prefix_end(const Ctx &c, PrefixAcc &a, const StateDev &st, kdss_result *out);
void fw_run_external(const Ctx &c, const SctDev &s, uint64_t *r, uint64_t *acc, int32_t *slow,
                     int *slow_count, int *err, unsigned long long *maxr, int T);
// Prefix-shared SCTs (share.cu): encoding of a flat SCT, c_k at k, states,
// synchronous iterations and extraction chunk by chunk, and a full decode.
void fc_encode(const Ctx &c, const SctDev &s, int64_t chunk_pairs, FcDev &fc);
void fc_ck_at(const Ctx &c, const SctDev &meta, const FcDev &fc, int k, uint64_t &lo, uint64_t &hi);
void fc_state_init(const Ctx &c, const SctDev &meta, const FcDev &fc, int k, int precision, StateDev &st);
void fc_iterate(const Ctx &c, const SctDev &meta, const FcDev &fc, StateDev &st, int T, bool profile);
void fc_extract(const Ctx &c, const SctDev &meta, const FcDev &fc, const StateDev &st, kdss_result *out);
void fc_decode_all(const Ctx &c, const SctDev &meta, const FcDev &fc, SctDev &out);

}  // namespace kdss
