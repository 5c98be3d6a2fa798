// fw.cu -- steps A4-A5: Frank-Wolfe iterations of PBUpdate over all pairs.
//
// Alg. 2 runs PBUpdate (Alg. 3) for every SCT pair in every iteration.  Here
// all pairs of iteration t read r_{t-1} (synchronous form: the per-pair
// allocations do not depend on the pair order, so integer sums are exact and
// reproducible) and scatter-add their allocation into a delta vector; the
// step kernel then forms r_t = r_{t-1} + delta.  With the cumulative r the FW
// iterate is r / t (step size 1/t, Sec. 3.3).
//
// PBUpdate of one pair (Alg. 3): n_C = C(p, k-h) units; V_h nodes may take up
// to C(p, k-h), V_p nodes up to C(p-1, k-h-1) (C3-C4 of SCT-CP, Lemma 2.6).
// Starting from the lowest plateau of r, the current plateau is raised by
// w = min(smallest remaining cap, gap to the next plateau, floor(n_C/|V_i|))
// (line 10); capped nodes leave (line 18); a plateau that reaches the next
// one merges with it (line 19); when floor(n_C/|V_i|) = 0 the remaining
// units go one each to the lowest-id nodes of the plateau (lines 15-17, with
// "random" read as "lowest id").  Nodes with zero cap never take part.
//
// GPU mapping: a pair is handled by a group of G lanes (G = 8 or 32 by length
// class), each lane holding NPL node slots in registers; node j of the pair
// sits in slot j / G of lane j % G.  Nodes are stored ascending by id, so
// "lowest id" is "lowest slot index" and the remainder ranks come from
// ballots.  Plateau levels, counts and caps are group reductions by
// butterfly shuffles.  Every loop runs warp-uniformly.
//
// The continuous rule (KDSS_FP32K) performs the same walk with real w and no
// remainder on the normalised iterate r/t: iteration t fills n_C / s units
// with caps cap / s on r_{t-1} / (t-1) (s = max(t-1, 1)), which equals the
// cumulative-scale fill divided by s; the allocation is summed with
// error-free (TwoSum) compensated atomics and folded into r/t by a Kahan
// update in the step kernel.
#include <algorithm>

#include "fw.cuh"

namespace kdss {

namespace {

constexpr int FW_THREADS = 256;
constexpr unsigned FULL = 0xffffffffu;

template <int G>
__device__ __forceinline__ uint64_t gmin_u64(uint64_t v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        uint64_t t = __shfl_xor_sync(FULL, v, o);
        v = t < v ? t : v;
    }
    return v;
}
template <int G>
__device__ __forceinline__ float gmin_f32(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(FULL, v, o));
    return v;
}
template <int G>
__device__ __forceinline__ int gsum_i32(int v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <class RT>
__device__ __forceinline__ uint64_t load_r(const RT *r, int32_t id);
template <>
__device__ __forceinline__ uint64_t load_r<uint64_t>(const uint64_t *r, int32_t id) {
    return __ldg(r + id);
}
template <>
__device__ __forceinline__ uint64_t load_r<double>(const double *r, int32_t id) {
    return (uint64_t)__ldg(r + id);
}
__device__ __forceinline__ void add_acc(uint64_t *acc, int32_t id, uint64_t d) {
    atomicAdd((unsigned long long *)(acc + id), (unsigned long long)d);
}
__device__ __forceinline__ void add_acc(double *acc, int32_t id, uint64_t d) {
    atomicAdd(acc + id, (double)d);
}

// Rule I (integer) PBUpdate over the pairs [p_begin, p_end).
template <int G, int NPL, class RT>
__global__ void __launch_bounds__(FW_THREADS)
k_pbupdate_int(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
               const uint8_t *__restrict__ hcnt, int64_t p_begin, int64_t p_end,
               const RT *__restrict__ r, RT *acc, const uint64_t *__restrict__ binom, int bcols,
               int k, int *err) {
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned lowmask = (G == 32) ? FULL : ((1u << G) - 1u);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t np = p_end - p_begin;
    for (int64_t wb = warp * GPW; wb < np; wb += nwarps * GPW) {
        const int64_t qi = wb + lane / G;
        const bool active = qi < np;
        const int64_t q = p_begin + qi;
        int64_t off0 = 0;
        int len = 0, h = 0;
        if (active) {
            off0 = pair_off[q];
            len = (int)(pair_off[q + 1] - off0);
            h = hcnt[q];
        }
        const int p = len - h;
        uint64_t nC = 0, cap_h = 0, cap_p = 0;
        if (active) {
            nC = __ldg(binom + (size_t)p * bcols + (k - h));
            cap_h = nC;
            cap_p = (p >= 1 && k - h - 1 >= 0) ? __ldg(binom + (size_t)(p - 1) * bcols + (k - h - 1)) : 0ull;
        }
        uint64_t r0[NPL], cur[NPL], up[NPL];
        int32_t id[NPL];
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int j = s * G + gl;
            const bool valid = active && j < len;
            const int32_t raw = valid ? __ldg(nodes + off0 + j) : 0;
            id[s] = raw & 0x7fffffff;
            r0[s] = valid ? load_r<RT>(r, id[s]) : ~0ull;
            up[s] = valid ? (raw < 0 ? cap_h : cap_p) : 0ull;
            cur[s] = r0[s];
        }
        uint64_t rem = active ? nC : 0ull;
        uint64_t lev;
        {
            uint64_t m = ~0ull;
#pragma unroll
            for (int s = 0; s < NPL; ++s)
                if (up[s] > 0 && cur[s] < m) m = cur[s];
            lev = gmin_u64<G>(m);
        }
        int guard = 0;
        const int guard_max = 4 * G * NPL + 8;
        while (__any_sync(FULL, rem > 0)) {
            uint64_t nx = ~0ull, mu = ~0ull;
            int na = 0;
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                if (up[s] > 0) {
                    if (cur[s] == lev) { ++na; mu = up[s] < mu ? up[s] : mu; }
                    else if (cur[s] > lev && cur[s] < nx) nx = cur[s];
                }
            }
            na = gsum_i32<G>(na);
            mu = gmin_u64<G>(mu);
            nx = gmin_u64<G>(nx);
            bool do_rem = false;
            if (rem > 0) {
                if (na == 0) {
                    if (nx == ~0ull) { atomicOr(err, DERR_LOGIC); rem = 0; }
                    else lev = nx;
                } else {
                    const uint64_t gap = nx == ~0ull ? ~0ull : nx - lev;
                    uint64_t w = mu < gap ? mu : gap;
                    const uint64_t share = rem / (uint64_t)na;
                    w = share < w ? share : w;
                    if (w > 0) {
#pragma unroll
                        for (int s = 0; s < NPL; ++s)
                            if (up[s] > 0 && cur[s] == lev) { cur[s] += w; up[s] -= w; }
                        rem -= w * (uint64_t)na;
                        lev += w;
                    } else {
                        do_rem = true;
                    }
                }
            }
            if (__any_sync(FULL, do_rem)) {
                int before = 0;
#pragma unroll
                for (int s = 0; s < NPL; ++s) {
                    const bool inA = do_rem && up[s] > 0 && cur[s] == lev;
                    const unsigned gb = (__ballot_sync(FULL, inA) >> gbase) & lowmask;
                    const int rk = before + __popc(gb & ((1u << gl) - 1u));
                    if (inA && (uint64_t)rk < rem) { cur[s] += 1; up[s] -= 1; }
                    before += __popc(gb);
                }
                if (do_rem) rem = 0;
            }
            if (++guard > guard_max) {
                if (rem > 0) atomicOr(err, DERR_LOGIC);
                break;
            }
        }
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int j = s * G + gl;
            if (active && j < len && cur[s] > r0[s]) add_acc(acc, id[s], cur[s] - r0[s]);
        }
    }
}

// Rule C (continuous) PBUpdate on the normalised iterate, FP32.
template <int G, int NPL>
__global__ void __launch_bounds__(FW_THREADS)
k_pbupdate_f32(const int64_t *__restrict__ pair_off, const int32_t *__restrict__ nodes,
               const uint8_t *__restrict__ hcnt, int64_t p_begin, int64_t p_end,
               const float *__restrict__ r, float *acc, float *accc,
               const uint64_t *__restrict__ binom, int bcols, int k, float inv_sigma, int *err) {
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t np = p_end - p_begin;
    const float INF = __int_as_float(0x7f800000);
    for (int64_t wb = warp * GPW; wb < np; wb += nwarps * GPW) {
        const int64_t qi = wb + lane / G;
        const bool active = qi < np;
        const int64_t q = p_begin + qi;
        int64_t off0 = 0;
        int len = 0, h = 0;
        if (active) {
            off0 = pair_off[q];
            len = (int)(pair_off[q + 1] - off0);
            h = hcnt[q];
        }
        const int p = len - h;
        float nC = 0.f, cap_h = 0.f, cap_p = 0.f;
        if (active) {
            nC = (float)__ldg(binom + (size_t)p * bcols + (k - h)) * inv_sigma;
            cap_h = nC;
            cap_p = (p >= 1 && k - h - 1 >= 0)
                        ? (float)__ldg(binom + (size_t)(p - 1) * bcols + (k - h - 1)) * inv_sigma
                        : 0.f;
        }
        float r0[NPL], cur[NPL], up[NPL];
        int32_t id[NPL];
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int j = s * G + gl;
            const bool valid = active && j < len;
            const int32_t raw = valid ? __ldg(nodes + off0 + j) : 0;
            id[s] = raw & 0x7fffffff;
            r0[s] = valid ? __ldg(r + id[s]) : INF;
            up[s] = valid ? (raw < 0 ? cap_h : cap_p) : 0.f;
            cur[s] = r0[s];
        }
        float rem = active ? nC : 0.f;
        float lev;
        {
            float m = INF;
#pragma unroll
            for (int s = 0; s < NPL; ++s)
                if (up[s] > 0.f) m = fminf(m, cur[s]);
            lev = gmin_f32<G>(m);
        }
        int guard = 0;
        const int guard_max = 4 * G * NPL + 8;
        while (__any_sync(FULL, rem > 0.f)) {
            float nx = INF, mu = INF;
            int na = 0;
#pragma unroll
            for (int s = 0; s < NPL; ++s) {
                if (up[s] > 0.f) {
                    if (cur[s] == lev) { ++na; mu = fminf(mu, up[s]); }
                    else if (cur[s] > lev) nx = fminf(nx, cur[s]);
                }
            }
            na = gsum_i32<G>(na);
            mu = gmin_f32<G>(mu);
            nx = gmin_f32<G>(nx);
            if (rem > 0.f) {
                if (na == 0) {
                    if (nx == INF) { atomicOr(err, DERR_LOGIC); rem = 0.f; }
                    else lev = nx;
                } else {
                    const float gap = nx - lev;
                    const float share = rem / (float)na;
                    float w = fminf(mu, gap);
                    const bool last = share <= w;
                    if (last) w = share;
                    const float nl = (!last && w == gap) ? nx : lev + w;
#pragma unroll
                    for (int s = 0; s < NPL; ++s)
                        if (up[s] > 0.f && cur[s] == lev) { cur[s] = nl; up[s] -= w; }
                    rem = last ? 0.f : rem - w * (float)na;
                    if (rem < 0.f) rem = 0.f;
                    lev = nl;
                }
            }
            if (++guard > guard_max) break;
        }
#pragma unroll
        for (int s = 0; s < NPL; ++s) {
            const int j = s * G + gl;
            if (active && j < len && cur[s] > r0[s]) {
                const float x = cur[s] - r0[s];
                const float old = atomicAdd(acc + id[s], x);
                // TwoSum: exact rounding error of the sum the atomic stored
                const float sum = old + x;
                const float bp = sum - old;
                const float e = (old - (sum - bp)) + (x - bp);
                if (e != 0.f) atomicAdd(accc + id[s], e);
            }
        }
    }
}

// r_t = r_{t-1} + delta (rule I); running max of r for the bound.
template <class RT>
__global__ void k_step_int(int64_t n, RT *r, RT *acc, unsigned long long *maxr) {
    unsigned long long m = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        RT x = r[v] + acc[v];
        r[v] = x;
        acc[v] = RT(0);
        unsigned long long b;
        if constexpr (sizeof(RT) == 8 && RT(0.5) != RT(0)) b = (unsigned long long)__double_as_longlong((double)x);
        else b = (unsigned long long)x;
        m = b > m ? b : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(FULL, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(maxr, m);
}

// rhat_t = rhat_{t-1} + (s * a - rhat_{t-1}) / t with Kahan compensation.
__global__ void k_step_f32(int64_t n, float *r, float *rc, float *a, float *ac, float sigma,
                           float inv_t) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const float delta = sigma * (a[v] + ac[v]);
        const float rv = r[v];
        const float y = (delta - rv) * inv_t - rc[v];
        const float tt = rv + y;
        rc[v] = (tt - rv) - y;
        r[v] = tt;
        a[v] = 0.f;
        ac[v] = 0.f;
    }
}

template <class RT>
void launch_int_class(const Ctx &c, const SctDev &s, int cls, RT *r, RT *acc, int *err) {
    const int64_t b = s.class_begin[cls], e = s.class_begin[cls + 1];
    if (e <= b) return;
    const int64_t np = e - b;
    const int bc = s.k + 1;
    auto go = [&](auto kern, int G) {
        const int64_t groups_per_block = (FW_THREADS / 32) * (32 / G);
        int grid = (int)std::min<int64_t>(ceil_div(np, groups_per_block), (int64_t)c.num_sms * 16);
        kern<<<grid, FW_THREADS, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, b, e, r, acc,
                                                s.binom.p, bc, s.k, err);
        KDSS_LAUNCH_CHECK();
    };
    switch (cls) {
        case 0: go(k_pbupdate_int<8, 1, RT>, 8); break;
        case 1: go(k_pbupdate_int<8, 2, RT>, 8); break;
        case 2: go(k_pbupdate_int<8, 4, RT>, 8); break;
        case 3: go(k_pbupdate_int<32, 8, RT>, 32); break;
        default: go(k_pbupdate_int<32, 32, RT>, 32); break;
    }
}

void launch_f32_class(const Ctx &c, const SctDev &s, int cls, StateDev &st, float inv_sigma) {
    const int64_t b = s.class_begin[cls], e = s.class_begin[cls + 1];
    if (e <= b) return;
    const int64_t np = e - b;
    const int bc = s.k + 1;
    auto go = [&](auto kern, int G) {
        const int64_t groups_per_block = (FW_THREADS / 32) * (32 / G);
        int grid = (int)std::min<int64_t>(ceil_div(np, groups_per_block), (int64_t)c.num_sms * 16);
        kern<<<grid, FW_THREADS, 0, c.stream>>>(s.pair_off.p, s.nodes.p, s.h.p, b, e, st.r32.p,
                                                st.a32.p, st.a32c.p, s.binom.p, bc, s.k,
                                                inv_sigma, st.err.p);
        KDSS_LAUNCH_CHECK();
    };
    switch (cls) {
        case 0: go(k_pbupdate_f32<8, 1>, 8); break;
        case 1: go(k_pbupdate_f32<8, 2>, 8); break;
        case 2: go(k_pbupdate_f32<8, 4>, 8); break;
        case 3: go(k_pbupdate_f32<32, 8>, 32); break;
        default: go(k_pbupdate_f32<32, 32>, 32); break;
    }
}

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};

}  // namespace

void fw_init(const Ctx &c, const SctDev &s, int precision, StateDev &st) {
    st.precision = precision;
    st.n = s.n;
    st.t = 0;
    st.ctx = c;
    const size_t n = (size_t)std::max<int64_t>(s.n, 1);
    if (precision == KDSS_FP32K) {
        st.r32 = DBuf<float>(c, n);
        st.r32c = DBuf<float>(c, n);
        st.a32 = DBuf<float>(c, n);
        st.a32c = DBuf<float>(c, n);
        zero(c, st.r32.p, n * 4);
        zero(c, st.r32c.p, n * 4);
        zero(c, st.a32.p, n * 4);
        zero(c, st.a32c.p, n * 4);
    } else {
        st.r = DBuf<uint64_t>(c, n);
        st.acc = DBuf<uint64_t>(c, n);
        zero(c, st.r.p, n * 8);
        zero(c, st.acc.p, n * 8);
    }
    st.maxr = DBuf<unsigned long long>(c, 1);
    st.err = DBuf<int>(c, 1);
    zero(c, st.maxr.p, 8);
    zero(c, st.err.p, 4);
}

void fw_run(const Ctx &c, const SctDev &s, StateDev &st, int T, bool profile) {
    if (T <= 0) return;
    const int64_t n = s.n;
    // exactness of the cumulative r: r_t(u) <= t * c_k
    if (st.precision != KDSS_FP32K) {
        const long double lim = st.precision == KDSS_INT64 ? 9.2e18L : 9.007199254740992e15L;
        const long double ck = (long double)s.ck_lo + (long double)s.ck_hi * 18446744073709551616.0L;
        if ((long double)(st.t + T) * ck >= lim)
            fail(KDSS_ERR_OVERFLOW, "T * c_k leaves the exact range of r");
    }
    std::vector<EventPair> ev;
    if (profile) ev.resize((size_t)T * 2);
    auto rec = [&](cudaEvent_t &e) {
        KDSS_CUDA(cudaEventCreate(&e));
        KDSS_CUDA(cudaEventRecord(e, c.stream));
    };
    const int B = 256;
    const int sgrid = grid_for(c, n, B, 4);
    for (int it = 0; it < T; ++it) {
        const int t = st.t + 1;  // iteration number, 1-based
        if (profile) rec(ev[2 * it].a);
        if (st.precision == KDSS_FP32K) {
            const float inv_sigma = (float)(1.0 / (double)std::max(t - 1, 1));
            for (int cl = 0; cl < NCLASS; ++cl) launch_f32_class(c, s, cl, st, inv_sigma);
        } else if (st.precision == KDSS_FP64) {
            for (int cl = 0; cl < NCLASS; ++cl)
                launch_int_class<double>(c, s, cl, (double *)st.r.p, (double *)st.acc.p, st.err.p);
        } else {
            for (int cl = 0; cl < NCLASS; ++cl)
                launch_int_class<uint64_t>(c, s, cl, st.r.p, st.acc.p, st.err.p);
        }
        if (profile) { rec(ev[2 * it].b); rec(ev[2 * it + 1].a); }
        if (n > 0) {
            if (st.precision == KDSS_FP32K) {
                const double sigma = (double)std::max(t - 1, 1);
                k_step_f32<<<sgrid, B, 0, c.stream>>>(n, st.r32.p, st.r32c.p, st.a32.p, st.a32c.p,
                                                     (float)sigma, (float)(1.0 / (double)t));
            } else if (st.precision == KDSS_FP64) {
                k_step_int<double><<<sgrid, B, 0, c.stream>>>(n, (double *)st.r.p, (double *)st.acc.p,
                                                              st.maxr.p);
            } else {
                k_step_int<uint64_t><<<sgrid, B, 0, c.stream>>>(n, st.r.p, st.acc.p, st.maxr.p);
            }
            KDSS_LAUNCH_CHECK();
        }
        if (profile) rec(ev[2 * it + 1].b);
        st.t = t;
    }
    int herr = 0;
    to_host(c, &herr, st.err.p, 1);
    if (profile) {
        for (int it = 0; it < T; ++it) {
            float a = 0.f, b2 = 0.f;
            KDSS_CUDA(cudaEventElapsedTime(&a, ev[2 * it].a, ev[2 * it].b));
            KDSS_CUDA(cudaEventElapsedTime(&b2, ev[2 * it + 1].a, ev[2 * it + 1].b));
            st.timing.fw_kernel_ms += a;
            st.timing.step_kernel_ms += b2;
            st.timing.fw_launches += 1;
            st.timing.step_launches += 1;
        }
        for (auto &e : ev) {
            cudaEventDestroy(e.a);
            cudaEventDestroy(e.b);
        }
    }
    if (herr) fail(KDSS_ERR_CUDA, "FW iteration: water-filling invariant failed on the device");
}

}  // namespace kdss
