// graph.cuh -- device-resident graph of the solver (steps A1-A2).
#pragma once

#include "kdss_internal.cuh"

namespace kdss {

struct GraphDev {
    int64_t n = 0;
    int64_t nadj = 0;             // 2 m entries of the symmetric CSR
    DBuf<int64_t> off;            // [n + 1], original ids
    DBuf<int32_t> adj;            // [2 m], neighbours ascending
    DBuf<int32_t> core;           // [n] core number
    DBuf<int32_t> rnd;            // [n] peel round
    DBuf<int32_t> rank;           // [n] position of v in the build order
    DBuf<int32_t> vert;           // [n] vertex at position i
    DBuf<int64_t> out_off;        // [n + 1], indexed by rank
    DBuf<int32_t> out_adj;        // [m] later neighbours as ranks, ascending
    int degeneracy = 0;
    int max_out = 0;
    int64_t peel_rounds = 0;
};

// Steps A1-A2: CSR of the simple graph, core numbers / peel rounds, the
// vertex order (KDSS_ORDER_*) and the oriented out-CSR in rank space.
void build_graph(const Ctx &c, const kdss_graph_desc &g, int order, GraphDev &out);

}  // namespace kdss
