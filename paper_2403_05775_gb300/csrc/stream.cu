// stream.cu -- the whole path for graphs whose SCT does not fit the device.
//
// Thm 3.7 puts the SCT at O(eta) space, and a dense core makes eta far larger
// than the graph.  In the synchronous form every pair of iteration t reads
// r_{t-1} and only the sum of the allocations matters, so the pairs can be
// visited in any grouping: the roots (in the build order) are split into
// ranges, and each iteration rebuilds the SCT of one range at a time (the
// per-root recursion of step A3 restricted to those roots), runs PBUpdate on
// it into the shared delta, and frees it before the next range; the step
// then closes the iteration.  The integer sums are exact, so r_T equals the
// unsplit iterations bit for bit.  Extraction visits the ranges the same way:
// the prefix-count increments of each range's pairs are added into the same
// histograms.  Memory holds the graph, r, and one range's pairs at a time;
// the price is one SCT build per range and iteration.
#include <algorithm>
#include <cstring>

#include "handles.cuh"

namespace kdss {

void fw_step_advance(const Ctx &c, StateDev &st, int64_t n);

namespace {

struct Chunks {
    int64_t n = 0;
    int count = 1;
    int64_t lo(int i) const { return n * i / count; }
    int64_t hi(int i) const { return n * (i + 1) / count; }
};

}  // namespace

void solve_streamed(const Ctx &c, const kdss_graph_desc &g, int k, int T, int nchunks, int precision,
                    int order, kdss_result *out) {
    memset(out, 0, sizeof *out);
    out->T = T;
    GraphDev gd;
    build_graph(c, g, order, gd);
    const int64_t n = gd.n;
    gd.off.reset();
    gd.adj.reset();
    Chunks ch;
    ch.n = n;
    ch.count = (int)std::max<int64_t>(1, std::min<int64_t>(nchunks, std::max<int64_t>(n, 1)));
    // sizing pass: c_k and the largest short-pair count over the ranges
    uint64_t ck_lo = 0, ck_hi = 0;
    int64_t short_max = 1;
    for (int i = 0; i < ch.count; ++i) {
        SctDev s;
        build_sct(c, gd, k, s, -1, ch.lo(i), ch.hi(i));
        const uint64_t o = ck_lo;
        ck_lo += s.ck_lo;
        ck_hi += s.ck_hi + (ck_lo < o ? 1ull : 0ull);
        short_max = std::max<int64_t>(short_max, s.class_begin[3] - s.class_begin[0]);
    }
    if (precision != KDSS_FP32K) {
        const long double lim = precision == KDSS_INT64 ? 9.2e18L : 9.007199254740992e15L;
        const long double ck = (long double)ck_lo + (long double)ck_hi * 18446744073709551616.0L;
        if ((long double)T * ck >= lim) fail(KDSS_ERR_OVERFLOW, "T * c_k leaves the exact range of r");
    }
    StateDev st;
    fw_init_n(c, n, short_max, precision, st);
    for (int t = 0; t < T; ++t) {
        for (int i = 0; i < ch.count; ++i) {
            SctDev s;
            build_sct(c, gd, k, s, -1, ch.lo(i), ch.hi(i));
            if (s.npairs > 0) fw_enqueue_group(c, s, st, 0);
            sync(c);   // the range's pairs are freed when s goes out of scope
        }
        fw_step_advance(c, st, n);
    }
    int herr = 0;
    to_host(c, &herr, st.err.p, 1);
    if (herr) fail(KDSS_ERR_CUDA, "FW iteration: water-filling invariant failed on the device");
    if (n == 0) {
        out->t_used = T;
        return;
    }
    PrefixAcc a;
    prefix_begin(c, n, st, ck_hi != 0, a);
    for (int i = 0; i < ch.count; ++i) {
        SctDev s;
        build_sct(c, gd, k, s, -1, ch.lo(i), ch.hi(i));
        if (s.npairs > 0) prefix_add(c, s, k, a);
        sync(c);
    }
    prefix_end(c, a, st, out);
    out->T = T;
    out->t_used = T;
}

}  // namespace kdss
