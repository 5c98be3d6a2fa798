// fw.cuh -- Frank-Wolfe state and iterations (steps A4-A5).
#pragma once

#include <functional>

#include "sct.cuh"

namespace kdss {

struct StateDev {
    int precision = KDSS_INT64;
    int64_t n = 0;
    int t = 0;                       // iterations done
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

void fw_init(const Ctx &c, const SctDev &s, int precision, StateDev &st);
void fw_run(const Ctx &c, const SctDev &s, StateDev &st, int T, bool profile);
// in-place (asynchronous) iterations of the integer rule: pairs add into r
void fw_run_async(const Ctx &c, const SctDev &s, StateDev &st, int T);
void fw_enqueue_inplace(const Ctx &c, const SctDev &s, StateDev &st);
// batches: several SCTs over disjoint node ranges of one state
void fw_init_n(const Ctx &c, int64_t n, int64_t short_capacity, int precision, StateDev &st);
void fw_enqueue_group(const Ctx &c, const SctDev &s, StateDev &st, int64_t node_off);
void fw_enqueue_step_range(const Ctx &c, StateDev &st, int64_t node_off, int64_t n, bool advance);
long long fw_capture(const Ctx &c, cudaGraphExec_t *exec, const std::function<void(const Ctx &)> &fn);
void fw_run_external(const Ctx &c, const SctDev &s, uint64_t *r, uint64_t *acc, int32_t *slow,
                     int *slow_count, int *err, unsigned long long *maxr, int T);

}  // namespace kdss
