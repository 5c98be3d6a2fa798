// share.cu -- the prefix-shared form of an SCT (Sec. 2, Lemmas 2.4-2.5).
//
// The pairs of one recursion share the hold and pivot nodes of the branch
// they come from, so their node lists repeat long prefixes.  The shared form
// keeps every prefix once: within each length class the pairs are sorted in
// lexicographic order of their node words (ids ascending, HOLD_BIT on V_h
// nodes, so V_h and V_p members of the same id differ), and a pair keeps only
// the words after the longest prefix it shares with the pair before it
// (front coding: the kept words of a sorted list are exactly the nodes of its
// prefix tree).  Every block of FC_BLOCK pairs starts with a pair kept whole,
// so that a warp decodes a block on its own, a lane per pair.
//
// The FW iterations and the extraction take chunks of whole blocks, decode
// each into the flat layout (pair offsets, node words, h) in a scratch SCT
// and run the same PBUpdate kernels on it: in the synchronous form all pairs
// of iteration t read r_{t-1} and only the sum of the allocations matters,
// so r_T equals the flat form's bit for bit.  The device keeps the shared
// form, the scratch of one chunk, the graph-free counts and the binomial
// tables; the flat pair stream exists one chunk at a time.
#include <algorithm>
#include <cstring>

#include "handles.cuh"

namespace kdss {

void fw_step_advance(const Ctx &c, StateDev &st, int64_t n);

namespace {

// Position i of the shared order holds pair perm[i]: its length, h and the
// prefix it shares with the pair at i - 1 (0 at the start of a block).
// blk_first[i] != 0 marks the first pair of a block.
__global__ void k_fc_lcp(int64_t np, const int32_t *__restrict__ perm,
                         const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
                         const uint8_t *__restrict__ h_in, const uint8_t *__restrict__ blk_first,
                         uint16_t *lcp, uint16_t *len, uint8_t *h_out, int64_t *kept,
                         int64_t *flat) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = perm[i];
        const int64_t o = pair_off[q];
        const int l = (int)(pair_off[q + 1] - o);
        int m = 0;
        if (!blk_first[i]) {
            const int64_t qp = perm[i - 1];
            const int64_t op = pair_off[qp];
            const int lp = (int)(pair_off[qp + 1] - op);
            const int lim = l < lp ? l : lp;
            while (m < lim && nodes[o + m] == nodes[op + m]) ++m;
        }
        lcp[i] = (uint16_t)m;
        len[i] = (uint16_t)l;
        h_out[i] = h_in[q];
        kept[i] = l - m;
        flat[i] = l;
    }
}

// The kept words of every pair: nodes[m, len) of pair perm[i] at word_off[i].
__global__ void k_fc_words(int64_t np, const int32_t *__restrict__ perm,
                           const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
                           const uint16_t *__restrict__ lcp, const int64_t *__restrict__ word_off,
                           uint32_t *words) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < np; i += nwarps) {
        const int64_t q = perm[i];
        const int64_t o = pair_off[q], l = pair_off[q + 1] - o;
        const int m = lcp[i];
        for (int64_t x = m + lane; x < l; x += 32) words[word_off[i] + (x - m)] = (uint32_t)nodes[o + x];
    }
}

// Block tables from the per-pair offsets: first kept word and first flat
// node of every block (and the ends, at nblocks).
__global__ void k_fc_blocks(int64_t nb, const int64_t *__restrict__ bpair,
                            const int64_t *__restrict__ word_off, const int64_t *__restrict__ flat_off,
                            int64_t np, int64_t nwords, int64_t nnodes, int64_t *bword, int64_t *bnode) {
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b <= nb;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = bpair[b];
        bword[b] = p < np ? word_off[p] : nwords;
        bnode[b] = p < np ? flat_off[p] : nnodes;
    }
}

// Decode blocks [b0, b1) into the flat layout of a scratch SCT: pair p
// (p0 <= p < p1) goes to slot p - p0, its nodes from flat node n0 on.  A warp
// per block, a lane per pair.  Word j of pair q was kept by the last pair
// q' <= q of the block whose kept words start at or before j (lcp[q'] <= j):
// every pair after q' up to q shares word j with the pair before it.
__global__ void k_fc_decode(int64_t b0, int64_t b1, const int64_t *__restrict__ bpair,
                            const int64_t *__restrict__ bword, const int64_t *__restrict__ bnode,
                            const uint16_t *__restrict__ lcp, const uint16_t *__restrict__ len,
                            const uint8_t *__restrict__ h, const uint32_t *__restrict__ words,
                            int64_t p0, int64_t n0, int64_t np_chunk, int64_t *pair_off,
                            int32_t *nodes, uint8_t *h_out) {
    const unsigned FULL_ = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned le = lanemask_lt() | (1u << lane);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = b0 + warp; b < b1; b += nwarps) {
        const int64_t pf = bpair[b], pe = bpair[b + 1];
        const int64_t q = pf + lane;
        const bool valid = q < pe;
        const int L = valid ? (int)len[q] : 0;
        const int P = valid ? (int)lcp[q] : 0x10000;   // never the owner of a word
        const int kept = valid ? L - P : 0;
        int ik = kept, iL = L;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int yk = __shfl_up_sync(FULL_, ik, o);
            const int yL = __shfl_up_sync(FULL_, iL, o);
            if (lane >= o) {
                ik += yk;
                iL += yL;
            }
        }
        const int64_t wo = bword[b] + (ik - kept);        // this pair's first kept word
        const int64_t fo = bnode[b] + (iL - L) - n0;      // its first flat node in the chunk
        if (valid) {
            pair_off[q - p0] = fo;
            h_out[q - p0] = h[q];
        }
        const int maxL = (int)__reduce_max_sync(FULL_, (unsigned)L);
        for (int j = 0; j < maxL; ++j) {
            // lane 0 keeps its pair whole (lcp 0), so the mask is never empty
            const unsigned m = __ballot_sync(FULL_, P <= j) & le;
            const int owner = 31 - __clz(m);
            const int64_t ow = __shfl_sync(FULL_, wo, owner);
            const int oP = __shfl_sync(FULL_, P, owner);
            if (valid && j < L) nodes[fo + j] = (int32_t)__ldg(words + ow + (j - oP));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) pair_off[np_chunk] = bnode[b1] - n0;
}

// max pair length of pairs [pb, pe) as u64 words (for reduce_max_u64)
__global__ void k_fc_lens(int64_t pb, int64_t pe, const int64_t *__restrict__ pair_off, uint64_t *out) {
    for (int64_t i = pb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pe;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i - pb] = (uint64_t)(pair_off[i + 1] - pair_off[i]);
}

__global__ void k_iota32(int64_t n, int32_t *v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (int32_t)i;
}

// Lexicographic word order packed in few bits: (id << 1 | hold) + 1, 0 past
// the end.  Equal words give equal keys, so sorting on these keys groups
// the same prefixes as sorting on the raw words.
__global__ void k_fc_keys_packed(int64_t np, const int32_t *__restrict__ perm,
                                 const int64_t *__restrict__ pair_off,
                                 const int32_t *__restrict__ nodes, int p, uint64_t *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = perm[i];
        const int64_t o = pair_off[q], len = pair_off[q + 1] - o;
        uint64_t key = 0ull;
        if (p < len) {
            const uint32_t w = (uint32_t)nodes[o + p];
            key = ((((uint64_t)(w & 0x7fffffffu)) << 1) | (uint64_t)(w >> 31)) + 1ull;
        }
        keys[i] = key;
    }
}

__global__ void k_fc_first(int64_t np, int64_t c0, int64_t c1, int64_t c2, int64_t c3, int64_t c4,
                           uint8_t *first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cb = i >= c4 ? c4 : i >= c3 ? c3 : i >= c2 ? c2 : i >= c1 ? c1 : c0;
        first[i] = ((i - cb) % FC_BLOCK) == 0 ? 1 : 0;
    }
}

void copy_binom(const Ctx &c, const SctDev &from, SctDev &to) {
    to.binom = DBuf<uint64_t>(c, from.binom.n);
    to.binom128 = DBuf<U128>(c, from.binom128.n);
    to.binomf = DBuf<float>(c, from.binomf.n);
    if (from.binom.n)
        KDSS_CUDA(cudaMemcpyAsync(to.binom.p, from.binom.p, from.binom.bytes(), cudaMemcpyDeviceToDevice, c.stream));
    if (from.binom128.n)
        KDSS_CUDA(cudaMemcpyAsync(to.binom128.p, from.binom128.p, from.binom128.bytes(),
                                  cudaMemcpyDeviceToDevice, c.stream));
    if (from.binomf.n)
        KDSS_CUDA(cudaMemcpyAsync(to.binomf.p, from.binomf.p, from.binomf.bytes(), cudaMemcpyDeviceToDevice,
                                  c.stream));
    to.binom_rows = from.binom_rows;
}

}  // namespace

void fc_encode(const Ctx &c, const SctDev &s, int64_t chunk_pairs, FcDev &fc) {
    const int64_t np = s.npairs;
    if (np > INT32_MAX) fail(KDSS_ERR_UNSUPPORTED, "prefix sharing takes at most 2^31 - 1 pairs");
    if (!s.pair_off.p && np > 0) fail(KDSS_ERR_INVALID_ARG, "the SCT holds no flat pairs");
    fc.npairs = np;
    fc.nnodes = s.nnodes;
    const int B = 256;
    // blocks of FC_BLOCK pairs, restarted at every class start
    std::vector<int64_t> hb;
    for (int cl = 0; cl < NCLASS; ++cl)
        for (int64_t p = s.class_begin[cl]; p < s.class_begin[cl + 1]; p += FC_BLOCK) hb.push_back(p);
    fc.nblocks = (int64_t)hb.size();
    hb.push_back(np);
    fc.bpair = DBuf<int64_t>(c, hb.size());
    to_device(c, fc.bpair.p, hb.data(), hb.size());
    fc.lcp = DBuf<uint16_t>(c, (size_t)std::max<int64_t>(np, 1));
    fc.len = DBuf<uint16_t>(c, (size_t)std::max<int64_t>(np, 1));
    fc.h = DBuf<uint8_t>(c, (size_t)std::max<int64_t>(np, 1));
    fc.bword = DBuf<int64_t>(c, hb.size());
    fc.bnode = DBuf<int64_t>(c, hb.size());
    DBuf<int64_t> word_off(c, (size_t)std::max<int64_t>(np, 1)), flat_off(c, (size_t)std::max<int64_t>(np, 1));
    if (np > 0) {
        // lexicographic order of the pairs of each class: stable LSD radix
        // passes, last word first
        DBuf<int32_t> perm(c, (size_t)np);
        DBuf<uint64_t> keys(c, (size_t)np);
        k_iota32<<<grid_for(c, np, B), B, 0, c.stream>>>(np, perm.p);
        KDSS_LAUNCH_CHECK();
        const int kbits = bit_length((uint64_t)std::max<int64_t>(s.n, 1) * 2 + 2);
        for (int cl = 0; cl < NCLASS; ++cl) {
            const int64_t pb = s.class_begin[cl], pe = s.class_begin[cl + 1];
            if (pe - pb < 2) continue;
            k_fc_lens<<<grid_for(c, pe - pb, B), B, 0, c.stream>>>(pb, pe, s.pair_off.p, keys.p);
            KDSS_LAUNCH_CHECK();
            const int maxlen = (int)reduce_max_u64(c, keys.p, pe - pb);
            for (int pos = maxlen - 1; pos >= 0; --pos) {
                k_fc_keys_packed<<<grid_for(c, pe - pb, B), B, 0, c.stream>>>(pe - pb, perm.p + pb, s.pair_off.p,
                                                                             s.nodes.p, pos, keys.p);
                KDSS_LAUNCH_CHECK();
                radix_sort_u64(c, keys.p, perm.p + pb, pe - pb, {BitRange{0, kbits}});
            }
        }
        keys.reset();
        DBuf<uint8_t> first(c, (size_t)np);
        k_fc_first<<<grid_for(c, np, B), B, 0, c.stream>>>(np, s.class_begin[0], s.class_begin[1],
                                                         s.class_begin[2], s.class_begin[3],
                                                         s.class_begin[4], first.p);
        KDSS_LAUNCH_CHECK();
        DBuf<int64_t> kept(c, (size_t)np), flat(c, (size_t)np);
        k_fc_lcp<<<grid_for(c, np, B), B, 0, c.stream>>>(np, perm.p, s.pair_off.p, s.nodes.p, s.h.p, first.p,
                                                       fc.lcp.p, fc.len.p, fc.h.p, kept.p, flat.p);
        KDSS_LAUNCH_CHECK();
        fc.nwords = exclusive_scan_i64(c, kept.p, word_off.p, np);
        const int64_t nn = exclusive_scan_i64(c, flat.p, flat_off.p, np);
        if (nn != s.nnodes) fail(KDSS_ERR_CUDA, "prefix sharing: node count differs from the SCT's");
        fc.words = DBuf<uint32_t>(c, (size_t)fc.nwords + 1);
        k_fc_words<<<grid_for(c, np * 32, B), B, 0, c.stream>>>(np, perm.p, s.pair_off.p, s.nodes.p, fc.lcp.p,
                                                              word_off.p, fc.words.p);
        KDSS_LAUNCH_CHECK();
    } else {
        fc.words = DBuf<uint32_t>(c, 1);
    }
    k_fc_blocks<<<grid_for(c, fc.nblocks + 1, B), B, 0, c.stream>>>(fc.nblocks, fc.bpair.p, word_off.p,
                                                                  flat_off.p, np, fc.nwords, fc.nnodes,
                                                                  fc.bword.p, fc.bnode.p);
    KDSS_LAUNCH_CHECK();
    // chunks of whole blocks, up to chunk_pairs pairs each
    std::vector<int64_t> hn(hb.size());
    to_host(c, hn.data(), fc.bnode.p, hn.size());
    const int64_t per = std::max<int64_t>(FC_BLOCK, chunk_pairs);
    fc.chunks.clear();
    for (int64_t b = 0; b < fc.nblocks;) {
        int64_t e = b + 1;
        while (e < fc.nblocks && hb[e + 1] - hb[b] <= per) ++e;
        FcDev::Chunk ch{};
        ch.b0 = b;
        ch.b1 = e;
        ch.p0 = hb[b];
        ch.p1 = hb[e];
        ch.n0 = hn[b];
        ch.n1 = hn[e];
        for (int cl = 0; cl <= NCLASS; ++cl)
            ch.class_begin[cl] = std::min(std::max(s.class_begin[cl], ch.p0), ch.p1) - ch.p0;
        fc.max_chunk_pairs = std::max(fc.max_chunk_pairs, ch.p1 - ch.p0);
        fc.max_chunk_nodes = std::max(fc.max_chunk_nodes, ch.n1 - ch.n0);
        fc.max_chunk_short = std::max(fc.max_chunk_short, ch.class_begin[3] - ch.class_begin[0]);
        fc.chunks.push_back(ch);
        b = e;
    }
}

// The flat scratch SCT of one chunk at a time: the meta SCT's k, n and
// binomial tables, and pair arrays sized to the largest chunk.
void fc_scratch(const Ctx &c, const SctDev &meta, const FcDev &fc, SctDev &sc) {
    sc.k = meta.k;
    sc.n = meta.n;
    sc.max_len = meta.max_len;
    sc.ck_lo = meta.ck_lo;
    sc.ck_hi = meta.ck_hi;
    copy_binom(c, meta, sc);
    sc.pair_off = DBuf<int64_t>(c, (size_t)fc.max_chunk_pairs + 1);
    sc.nodes = DBuf<int32_t>(c, (size_t)fc.max_chunk_nodes + NODES_PAD);
    sc.h = DBuf<uint8_t>(c, (size_t)std::max<int64_t>(fc.max_chunk_pairs, 1));
    zero(c, sc.nodes.p, sc.nodes.bytes());
}

void fc_decode_chunk(const Ctx &c, const FcDev &fc, const FcDev::Chunk &ch, SctDev &sc) {
    const int64_t np = ch.p1 - ch.p0;
    sc.npairs = np;
    sc.nnodes = ch.n1 - ch.n0;
    for (int cl = 0; cl <= NCLASS; ++cl) sc.class_begin[cl] = ch.class_begin[cl];
    const int B = 256;
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(1, ceil_div(ch.b1 - ch.b0, B / 32)),
                                            (int64_t)c.num_sms * 8);
    k_fc_decode<<<grid, B, 0, c.stream>>>(ch.b0, ch.b1, fc.bpair.p, fc.bword.p, fc.bnode.p, fc.lcp.p,
                                          fc.len.p, fc.h.p, fc.words.p, ch.p0, ch.n0, np, sc.pair_off.p,
                                          sc.nodes.p, sc.h.p);
    KDSS_LAUNCH_CHECK();
}

// c_k at k (<= meta.k) of a shared k-agnostic SCT, chunk by chunk.
void fc_ck_at(const Ctx &c, const SctDev &meta, const FcDev &fc, int k, uint64_t &lo, uint64_t &hi) {
    if (k == meta.k) {
        lo = meta.ck_lo;
        hi = meta.ck_hi;
        return;
    }
    SctDev sc;
    fc_scratch(c, meta, fc, sc);
    lo = hi = 0;
    for (const auto &ch : fc.chunks) {
        fc_decode_chunk(c, fc, ch, sc);
        uint64_t l = 0, h = 0;
        sct_ck_at(c, sc, k, l, h);
        const uint64_t o = lo;
        lo += l;
        hi += h + (lo < o ? 1ull : 0ull);
    }
}

// A state for FW iterations at k over a shared SCT (r = 0, t = 0): its slow
// list holds the short pairs of the largest chunk.
void fc_state_init(const Ctx &c, const SctDev &meta, const FcDev &fc, int k, int precision, StateDev &st) {
    SctDev shell;
    shell.n = meta.n;
    shell.k = k;
    fc_ck_at(c, meta, fc, k, shell.ck_lo, shell.ck_hi);
    shell.class_begin[0] = 0;
    shell.class_begin[3] = fc.max_chunk_short;
    fw_init(c, shell, precision, st);
}

// T synchronous iterations: every chunk is decoded and updated from r_{t-1}
// into the shared delta, then the step closes the iteration.
void fc_iterate(const Ctx &c, const SctDev &meta, const FcDev &fc, StateDev &st, int T, bool profile) {
    if (st.precision != KDSS_FP32K) {
        const long double lim = st.precision == KDSS_INT64 ? 9.2e18L : 9.007199254740992e15L;
        const long double ck = (long double)st.ck_lo + (long double)st.ck_hi * 18446744073709551616.0L;
        if ((long double)(st.t + T) * ck >= lim) fail(KDSS_ERR_OVERFLOW, "(t + T) * c_k leaves the exact range of r");
    }
    if (T <= 0) return;
    SctDev sc;
    fc_scratch(c, meta, fc, sc);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (profile) {
        while (st.events.size() < 2) {
            cudaEvent_t e;
            KDSS_CUDA(cudaEventCreate(&e));
            st.events.push_back(e);
        }
        e0 = st.events[0];
        e1 = st.events[1];
        KDSS_CUDA(cudaEventRecord(e0, c.stream));
    }
    for (int t = 0; t < T; ++t) {
        for (const auto &ch : fc.chunks) {
            fc_decode_chunk(c, fc, ch, sc);
            fw_enqueue_group(c, sc, st, 0, st.k);
        }
        fw_step_advance(c, st, meta.n);
    }
    if (profile) KDSS_CUDA(cudaEventRecord(e1, c.stream));
    int herr = 0;
    to_host(c, &herr, st.err.p, 1);
    if (profile) {
        float ms = 0.f;
        KDSS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        st.timing.fw_kernel_ms += ms;
        st.timing.fw_launches += T;
    }
    if (herr) fail(KDSS_ERR_CUDA, "FW iteration: water-filling invariant failed on the device");
}

// Extraction (A6) with the prefix counts added chunk by chunk.
void fc_extract(const Ctx &c, const SctDev &meta, const FcDev &fc, const StateDev &st, kdss_result *out) {
    memset(out, 0, sizeof *out);
    out->t_used = st.t;
    if (meta.n == 0) return;
    SctDev sc;
    fc_scratch(c, meta, fc, sc);
    PrefixAcc a;
    prefix_begin(c, meta.n, st, st.ck_hi != 0, a);
    for (const auto &ch : fc.chunks) {
        fc_decode_chunk(c, fc, ch, sc);
        prefix_add(c, sc, st.k, a);
    }
    prefix_end(c, a, st, out);
}

// Every pair of the shared form, decoded into one flat SCT (for copies).
void fc_decode_all(const Ctx &c, const SctDev &meta, const FcDev &fc, SctDev &out) {
    FcDev::Chunk all{};
    all.b0 = 0;
    all.b1 = fc.nblocks;
    all.p0 = 0;
    all.p1 = fc.npairs;
    all.n0 = 0;
    all.n1 = fc.nnodes;
    for (int cl = 0; cl <= NCLASS; ++cl) all.class_begin[cl] = meta.class_begin[cl];
    FcDev one;
    one.max_chunk_pairs = fc.npairs;
    one.max_chunk_nodes = fc.nnodes;
    fc_scratch(c, meta, one, out);
    if (fc.nblocks > 0) fc_decode_chunk(c, fc, all, out);
    else to_device(c, out.pair_off.p, &fc.nnodes, 1);
    sync(c);
}

}  // namespace kdss
