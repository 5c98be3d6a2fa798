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
// Spare entries after the last node id of every SCT node array: the FW
// kernels copy id tiles widened to 16-byte boundaries.
constexpr int NODES_PAD = 4;

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
    DBuf<uint64_t> binom;         // C(a, b), a <= binom_rows - 1, b <= k; ~0 = 63 bits or more
    DBuf<U128> binom128;          // the same, exact below 2^128; U128_OVF beyond
    DBuf<float> binomf;           // the same rounded to float (the FP32 rule's counts)
    int binom_rows = 0;
    uint64_t ck_lo = 0, ck_hi = 0;
    int max_len = 0;
    int bcols() const { return k + 1; }   // columns of the binomial tables
    // Root-shared form of the same pairs (SCTs built here): every pair comes
    // from the recursion of one root, whose out-neighbourhood holds all its
    // nodes.  proot[q] is that root (rank); lidx[i] is node i of the pair as
    // an index into the root's neighbourhood list rnb_ids[rnb_off[root] ..]
    // (0 = the root itself, j + 1 = its j-th out-neighbour), bit 15 the V_h
    // mark, in the same slots as `nodes`.
    DBuf<int32_t> proot;          // [npairs]
    DBuf<uint16_t> lidx;          // [nnodes + NODES_PAD]
    DBuf<int64_t> rnb_off;        // [n + 1]
    DBuf<int32_t> rnb_ids;        // [n + out-edges] original ids
    bool rooted() const { return proot.p != nullptr; }
};

// Prefix-shared form of an SCT's pairs (front coding).  Within each length
// class the pairs are in lexicographic order of their node words (ids
// ascending, HOLD_BIT on V_h nodes), so pairs that share a prefix of nodes
// sit together; a pair keeps only the words after the prefix it shares with
// the pair before it, and every block of FC_BLOCK pairs (a warp, a lane per
// pair) starts with a pair kept whole.  The FW iterations and the
// extraction decode chunks of whole blocks into the flat layout of SctDev.
constexpr int FC_BLOCK = 32;
struct FcDev {
    int64_t npairs = 0, nnodes = 0, nwords = 0, nblocks = 0;
    DBuf<uint32_t> words;                  // [nwords + 1] the kept node words
    DBuf<uint16_t> lcp, len;               // [npairs] shared prefix, length
    DBuf<uint8_t> h;                       // [npairs] |V_h|
    DBuf<int64_t> bpair, bword, bnode;     // [nblocks + 1] first pair, first kept word,
                                           // first flat node of every block
    struct Chunk {
        int64_t b0, b1, p0, p1, n0, n1;    // blocks, pairs and flat nodes of the chunk
        int64_t class_begin[NCLASS + 1];   // relative to p0
    };
    std::vector<Chunk> chunks;
    int64_t max_chunk_pairs = 0, max_chunk_nodes = 0, max_chunk_short = 0;
    int64_t bytes() const {
        return (int64_t)(words.bytes() + lcp.bytes() + len.bytes() + h.bytes() + bpair.bytes() +
                         bword.bytes() + bnode.bytes());
    }
};

// Host tables of C(a, b) for a < rows, b <= k: in 64 bits (entries that need
// 63 bits or more hold ~0ull, treated as overflow by the integer kernels),
// in 128 bits (U128_OVF beyond) and rounded to float.
struct BinomTables {
    std::vector<uint64_t> t64;
    std::vector<U128> t128;
    std::vector<float> tf;
};
BinomTables host_binom_tables(int rows, int k);
std::vector<uint64_t> host_binom_table(int rows, int k);
// Bytes of an SCT's device tables and of its root-shared form.
inline int64_t binom_bytes(const SctDev &s) {
    return (int64_t)(s.binom.bytes() + s.binom128.bytes() + s.binomf.bytes() + s.proot.bytes() +
                     s.lidx.bytes() + s.rnb_off.bytes() + s.rnb_ids.bytes());
}

// klo < k: the k-agnostic form -- every pair with |V_h| <= k and at least
// klo nodes (the pruning of Lemma 2.5 for the sizes klo..k at once).
// The root-shared neighbourhood lists of every root (SctDev::rnb_*).
void build_root_neighbourhoods(const Ctx &c, const GraphDev &g, SctDev &out);
// root_lo / root_hi: only the pairs of the roots [root_lo, root_hi) in the
// build order (rank space); the default is every root.
void build_sct(const Ctx &c, const GraphDev &g, int k, SctDev &out, int klo = -1,
               int64_t root_lo = 0, int64_t root_hi = -1);
// P_k of a k-agnostic SCT: the pairs with |V_h| <= k <= |V(P)|, in order.
void sct_restrict(const Ctx &c, const SctDev &all, int k, SctDev &out);
// c_k of the pairs in P_k (|V_h| <= k <= |V(P)|) of an SCT built for k or, when
// k-agnostic, for every k up to its own; 128 bits.
void sct_ck_at(const Ctx &c, const SctDev &s, int k, uint64_t &lo, uint64_t &hi);
// Sizes of P_k from a count-only pass (nothing stored).  Counts cover the
// roots walked to the end; complete = 1 when that is every root.
constexpr int COUNT_MAX_OUT = 4095;
struct SctCount {
    int64_t eta = 0, L = 0;
    int64_t pairs_per_class[NCLASS + 1] = {};   // the last class: longer than 1024 nodes
    uint64_t ck_lo = 0, ck_hi = 0;
    int64_t roots_total = 0, roots_done = 0, roots_cut = 0, cut_pairs = 0, cut_nodes = 0;
    int max_len = 0, count_bits = 0, complete = 0;
    double seconds = 0;
};
void count_sct(const Ctx &c, const GraphDev &g, int k, double budget_s, SctCount &out);
void sct_from_pairs(const Ctx &c, int64_t n, int k, int64_t npairs, const int64_t *pair_off,
                    const int32_t *nodes, const int32_t *h, SctDev &out);

}  // namespace kdss
