// handles.cuh -- the opaque handle types of include/kdss.h.
#pragma once

#include "fw.cuh"

struct kdss_sct {
    kdss::Ctx ctx;
    kdss::GraphDev g;
    kdss::SctDev s;
    bool has_graph = false;
    int64_t m = 0;
    int degeneracy = 0;
    int max_out = 0;
    int kmax_multi = 0;           // > 0: a k-agnostic SCT for k <= kmax_multi (restrict first)
    kdss::DBuf<int32_t> cliques;  // explicit k-clique list (expanded on first use)
    int64_t nclq = -1;            // its length, -1 before expansion
    // prefix-shared form (kdss_sct_share_prefixes): the pairs live in `fc`;
    // `s` keeps the counts, classes and binomial tables, not the pairs
    bool shared = false;
    kdss::FcDev fc;
};

namespace kdss {
void expand_cliques(const Ctx &c, const SctDev &s, DBuf<int32_t> &out, int64_t &count);
void fw_cliques_run(const Ctx &c, const int32_t *cl, int64_t count, int k, StateDev &st, int T);
}  // namespace kdss

struct kdss_state {
    kdss::StateDev st;
};
