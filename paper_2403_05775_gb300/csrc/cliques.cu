// cliques.cu -- Alg. 1 over the explicit k-clique list, on the GPU.
//
// The paper's baseline form of the Frank-Wolfe step (Alg. 1): every k-clique
// hands its unit to its member of least (r, id).  The list is the expansion
// of the SCT: by Lemmas 2.4-2.5 pair (V_h, V_p) holds exactly the cliques
// V_h + S for the (k - |V_h|)-subsets S of V_p, each once.  Expansion: the
// clique counts n_C of the pairs are scanned into offsets; a warp per pair
// stages the pair's hold and pivot ids in shared memory, and each lane
// unranks clique j of the pair -- subset number j of V_p in the
// combinatorial number system (the largest x with C(x, i) <= j is the i-th
// element, for i = k - h down to 1).
//
// Iterations are synchronous (reading R1, as in fw.cu): every clique reads
// r_{t-1}; the units are aggregated per warp over equal receivers (cliques of
// one pair usually pick the same node) and added to a delta vector that the
// step kernel folds into r.  Integer sums: r_T equals the oracle's
// synchronous Alg. 1 exactly.
#include <cstring>

#include "handles.cuh"

namespace kdss {

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int EX_WARPS = 8;
constexpr int EX_MAXLEN = 1024;

__global__ void k_pair_nc(int64_t np, const int64_t *off, const uint8_t *h, const uint64_t *binom,
                          int bcols, int k, int64_t *nc) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < np;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int len = (int)(off[q + 1] - off[q]);
        const int hh = h[q];
        nc[q] = (int64_t)binom[(size_t)(len - hh) * bcols + (k - hh)];
    }
}

__global__ void __launch_bounds__(EX_WARPS * 32)
k_expand(int64_t np, const int64_t *__restrict__ off, const int32_t *__restrict__ nodes,
         const uint8_t *__restrict__ h, const uint64_t *__restrict__ binom, int bcols, int k,
         const int64_t *__restrict__ cbase, int32_t *out) {
    __shared__ int32_t sh[EX_WARPS][EX_MAXLEN];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t *hold = sh[wib];
    for (int64_t q = blockIdx.x * (int64_t)EX_WARPS + wib; q < np;
         q += (int64_t)gridDim.x * EX_WARPS) {
        const int64_t o0 = off[q];
        const int len = (int)(off[q + 1] - o0);
        const int hh = h[q];
        const int p = len - hh, m = k - hh;
        // hold ids first, pivot ids after them, both in stored (id) order
        int nh = 0, npv = 0;
        for (int b = 0; b < len; b += 32) {
            const int j = b + lane;
            const int32_t raw = j < len ? nodes[o0 + j] : 0;
            const bool isH = j < len && raw < 0, isP = j < len && raw >= 0;
            const unsigned mh = __ballot_sync(FULLM, isH), mp = __ballot_sync(FULLM, isP);
            const unsigned lt = (1u << lane) - 1u;
            if (isH) hold[nh + __popc(mh & lt)] = raw & 0x7fffffff;
            if (isP) hold[hh + npv + __popc(mp & lt)] = raw;
            nh += __popc(mh);
            npv += __popc(mp);
        }
        __syncwarp();
        const int32_t *piv = hold + hh;
        const uint64_t nC = binom[(size_t)p * bcols + m];
        const int64_t base = cbase[q];
        for (uint64_t j0 = lane; j0 < nC; j0 += 32) {
            int32_t *row = out + (size_t)(base + (int64_t)j0) * k;
            for (int t = 0; t < hh; ++t) row[t] = hold[t];
            uint64_t j = j0;
            int x = p;
            for (int i = m; i >= 1; --i) {
                // largest x' < x with C(x', i) <= j (C(i - 1, i) = 0 <= j ends it)
                do { --x; } while (binom[(size_t)x * bcols + i] > j);
                j -= binom[(size_t)x * bcols + i];
                row[hh + i - 1] = piv[x];
            }
        }
        __syncwarp();
    }
}

// one iteration of Alg. 1: every clique's unit to its member of least (r, id)
__global__ void k_alg1(int64_t c, const int32_t *__restrict__ cl, int k,
                       const uint64_t *__restrict__ r, unsigned long long *acc) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t b0 = blockIdx.x * (int64_t)blockDim.x; b0 < c; b0 += stride) {
        const int64_t q = b0 + threadIdx.x;
        int32_t best = -1;
        if (q < c) {
            const int32_t *C = cl + (size_t)q * k;
            best = C[0];
            uint64_t rb = __ldg(r + best);
            for (int j = 1; j < k; ++j) {
                const int32_t u = C[j];
                const uint64_t ru = __ldg(r + u);
                if (ru < rb || (ru == rb && u < best)) { best = u; rb = ru; }
            }
        }
        // aggregate equal receivers of the warp: one atomic per distinct node
        const unsigned act = __ballot_sync(FULLM, best >= 0);
        const unsigned same = __match_any_sync(FULLM, best);
        const unsigned mine = same & act;
        if (best >= 0 && lane == __ffs(mine) - 1)
            atomicAdd(acc + best, (unsigned long long)__popc(mine));
    }
}

__global__ void k_alg1_step(int64_t n, uint64_t *r, unsigned long long *acc,
                            unsigned long long *maxr) {
    unsigned long long m = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = r[v] + acc[v];
        r[v] = x;
        acc[v] = 0ull;
        m = x > m ? x : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(FULLM, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(maxr, m);
}

}  // namespace

void expand_cliques(const Ctx &c, const SctDev &s, DBuf<int32_t> &out, int64_t &count) {
    const int64_t np = s.npairs;
    const int k = s.k;
    count = 0;
    if (np == 0) {
        out = DBuf<int32_t>();
        return;
    }
    if (s.ck_hi) fail(KDSS_ERR_OVERFLOW, "more than 2^64 cliques");
    if (s.max_len > EX_MAXLEN) fail(KDSS_ERR_UNSUPPORTED, "a pair longer than 1024 nodes");
    const unsigned long long ck = s.ck_lo;
    size_t free_b = 0, total_b = 0;
    KDSS_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const long double need = (long double)ck * (long double)k * 4.0L;
    if (need > 0.5L * (long double)free_b) {
        char buf[240];
        snprintf(buf, sizeof buf,
                 "the explicit list of %llu %d-cliques needs %.1f GB, more than half of the "
                 "%.1f GB free (the SCT encodes them in %.3f GB)",
                 ck, k, (double)(need / 1e9L), 1e-9 * (double)free_b,
                 1e-9 * (double)(4 * s.nnodes + 9 * s.npairs));
        fail(KDSS_ERR_OOM, buf);
    }
    const int B = 256;
    DBuf<int64_t> nc(c, (size_t)np), base(c, (size_t)np);
    k_pair_nc<<<grid_for(c, np, B), B, 0, c.stream>>>(np, s.pair_off.p, s.h.p, s.binom.p, k + 1, k,
                                                      nc.p);
    KDSS_LAUNCH_CHECK();
    const int64_t total = exclusive_scan_i64(c, nc.p, base.p, np);
    if ((unsigned long long)total != ck) fail(KDSS_ERR_CUDA, "clique counts of the pairs do not add up to c_k");
    out = DBuf<int32_t>(c, (size_t)std::max<int64_t>(total * k, 1));
    const int grid = (int)std::min<int64_t>(ceil_div(np, EX_WARPS), (int64_t)c.num_sms * 8);
    k_expand<<<grid, EX_WARPS * 32, 0, c.stream>>>(np, s.pair_off.p, s.nodes.p, s.h.p, s.binom.p,
                                                   k + 1, k, base.p, out.p);
    KDSS_LAUNCH_CHECK();
    sync(c);
    count = total;
}

void fw_cliques_run(const Ctx &c, const int32_t *cl, int64_t count, int k, StateDev &st, int T) {
    if (T <= 0) return;
    if (st.precision != KDSS_INT64) fail(KDSS_ERR_UNSUPPORTED, "Alg. 1 iterations keep r in KDSS_INT64");
    if ((long double)(st.t + T) * (long double)count >= 9.2e18L)
        fail(KDSS_ERR_OVERFLOW, "T * c_k leaves the exact range of r");
    const int64_t n = st.n;
    const int B = 256;
    const int cgrid = grid_for(c, count, B, 8);
    const int sgrid = grid_for(c, n, B, 4);
    for (int it = 0; it < T; ++it) {
        if (count > 0) {
            k_alg1<<<cgrid, B, 0, c.stream>>>(count, cl, k, st.r.p, (unsigned long long *)st.acc.p);
            KDSS_LAUNCH_CHECK();
        }
        if (n > 0) {
            k_alg1_step<<<sgrid, B, 0, c.stream>>>(n, st.r.p, (unsigned long long *)st.acc.p,
                                                   st.maxr.p);
            KDSS_LAUNCH_CHECK();
        }
    }
    st.t += T;
}

}  // namespace kdss
