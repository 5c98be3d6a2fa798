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
};

struct kdss_state {
    kdss::StateDev st;
};
