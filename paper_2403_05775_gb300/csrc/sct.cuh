// sct.cuh -- device-resident SCT restricted to P_k (step A3).
#pragma once

#include "graph.cuh"

namespace kdss {

// Pairs are stored grouped by length class (the FW kernels use one
// thread-group shape per class); within a class, in root order then
// depth-first order.  A pair's nodes are ascending by id, bit 31 set on hold
// (V_h) nodes.
constexpr int NCLASS = 5;
constexpr int CLASS_MAXLEN[NCLASS] = {8, 16, 32, 256, 1024};
constexpr int MAX_PAIR_LEN = 1024;
constexpr uint32_t HOLD_BIT = 0x80000000u;

inline int pair_class(int len) {
    for (int c = 0; c < NCLASS; ++c)
        if (len <= CLASS_MAXLEN[c]) return c;
    return -1;
}

struct SctDev {
    int k = 0;
    int64_t n = 0;
    int64_t npairs = 0;
    int64_t nnodes = 0;
    DBuf<int64_t> pair_off;       // [npairs + 1]
    DBuf<int32_t> nodes;          // [nnodes]
    DBuf<uint8_t> h;              // [npairs] |V_h| (<= k <= 64)
    int64_t class_begin[NCLASS + 1] = {0, 0, 0, 0, 0, 0};
    DBuf<uint64_t> binom;         // C(a, b), a <= binom_rows - 1, b <= k; ~0 = overflow
    int binom_rows = 0;
    uint64_t ck_lo = 0, ck_hi = 0;
    int max_len = 0;
};

// Host table of C(a, b) for a < rows, b <= k in 64 bits; entries that need
// 63 bits or more hold ~0ull (treated as overflow by the kernels).
std::vector<uint64_t> host_binom_table(int rows, int k);

// klo < k: the k-agnostic form -- every pair with |V_h| <= k and at least
// klo nodes (the pruning of Lemma 2.5 for the sizes klo..k at once).
void build_sct(const Ctx &c, const GraphDev &g, int k, SctDev &out, int klo = -1);
// P_k of a k-agnostic SCT: the pairs with |V_h| <= k <= |V(P)|, in order.
void sct_restrict(const Ctx &c, const SctDev &all, int k, SctDev &out);
void sct_from_pairs(const Ctx &c, int64_t n, int k, int64_t npairs, const int64_t *pair_off,
                    const int32_t *nodes, const int32_t *h, SctDev &out);

}  // namespace kdss
