/* _rmat.c -- multi-threaded R-MAT draws, identical to synth.rmat's numpy path.
 *
 * Input generation only (no arithmetic of the solved method).  One block of
 * `cnt` draws: draw j descends `scale` levels; level l takes the uniform
 * (x >> 11) * 2^-53 of x = SplitMix64 output number base + j * scale + l of
 * the stream seeded with `sseed`, and picks quadrant a | b | c | d by the
 * thresholds a, a + b, a + b + c.  Draws with an endpoint >= n are dropped;
 * the accepted draws are written to src/dst in draw order and counted.
 */
#include <pthread.h>
#include <stdint.h>
#include <string.h>

#define GAMMA 0x9E3779B97F4A7C15ull

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

typedef struct {
    uint64_t sseed, base;
    int64_t lo, hi, n, kept;
    int scale;
    double a, ab, abc;
    int64_t *src, *dst;
} Job;

static void *run(void *p) {
    Job *J = (Job *)p;
    int64_t w = J->lo;
    for (int64_t j = J->lo; j < J->hi; ++j) {
        int64_t s = 0, d = 0;
        for (int l = 0; l < J->scale; ++l) {
            const uint64_t idx = J->base + (uint64_t)j * (uint64_t)J->scale + (uint64_t)l;
            const uint64_t x = mix64(J->sseed + (idx + 1ull) * GAMMA);
            const double u = (double)(x >> 11) * 0x1p-53;
            const int64_t bit = (int64_t)1 << (J->scale - 1 - l);
            const int right = (u >= J->a && u < J->ab) || u >= J->abc;
            const int down = u >= J->ab;
            if (down) s += bit;
            if (right) d += bit;
        }
        if (s < J->n && d < J->n) {
            J->src[w] = s;
            J->dst[w] = d;
            ++w;
        }
    }
    J->kept = w - J->lo;
    return NULL;
}

int64_t synth_rmat_block(uint64_t sseed, uint64_t base, int64_t cnt, int scale, double a, double ab,
                         double abc, int64_t n, int64_t *src, int64_t *dst, int nthreads) {
    enum { MAXT = 128 };
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MAXT) nthreads = MAXT;
    if (cnt < 4096) nthreads = 1;
    Job jobs[MAXT];
    pthread_t th[MAXT];
    int started[MAXT];
    for (int t = 0; t < nthreads; ++t) {
        Job *J = &jobs[t];
        J->sseed = sseed; J->base = base; J->scale = scale;
        J->a = a; J->ab = ab; J->abc = abc; J->n = n;
        J->lo = cnt * t / nthreads; J->hi = cnt * (t + 1) / nthreads;
        J->src = src; J->dst = dst; J->kept = 0;
        started[t] = t > 0 && pthread_create(&th[t], NULL, run, J) == 0;
    }
    run(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        else run(&jobs[t]);
    }
    int64_t w = jobs[0].kept;
    for (int t = 1; t < nthreads; ++t) {
        memmove(src + w, src + jobs[t].lo, (size_t)jobs[t].kept * sizeof(int64_t));
        memmove(dst + w, dst + jobs[t].lo, (size_t)jobs[t].kept * sizeof(int64_t));
        w += jobs[t].kept;
    }
    return w;
}

/* Chung-Lu endpoint draws, identical to synth.chung_lu's numpy path: draw j
 * takes the uniforms number j of the two streams (seeds sa, sb) and maps each
 * by inverse CDF: the count of cdf entries <= u (numpy searchsorted, side
 * 'right'), clipped to n - 1. */
typedef struct {
    uint64_t sa, sb;
    int64_t lo, hi, n;
    const double *cdf;
    int64_t *a, *b;
} CLJob;

static inline int64_t upper(const double *cdf, int64_t n, double u) {
    int64_t lo = 0, hi = n;  /* first index with cdf > u */
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (cdf[mid] <= u) lo = mid + 1; else hi = mid;
    }
    return lo < n - 1 ? lo : n - 1;
}

static void *run_cl(void *p) {
    CLJob *J = (CLJob *)p;
    for (int64_t j = J->lo; j < J->hi; ++j) {
        const uint64_t xa = mix64(J->sa + ((uint64_t)j + 1ull) * GAMMA);
        const uint64_t xb = mix64(J->sb + ((uint64_t)j + 1ull) * GAMMA);
        J->a[j] = upper(J->cdf, J->n, (double)(xa >> 11) * 0x1p-53);
        J->b[j] = upper(J->cdf, J->n, (double)(xb >> 11) * 0x1p-53);
    }
    return NULL;
}

void synth_chunglu_draws(uint64_t sa, uint64_t sb, int64_t m, const double *cdf, int64_t n,
                         int64_t *a, int64_t *b, int nthreads) {
    enum { MAXT = 128 };
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MAXT) nthreads = MAXT;
    if (m < 4096) nthreads = 1;
    CLJob jobs[MAXT];
    pthread_t th[MAXT];
    int started[MAXT];
    for (int t = 0; t < nthreads; ++t) {
        CLJob *J = &jobs[t];
        J->sa = sa; J->sb = sb; J->n = n; J->cdf = cdf; J->a = a; J->b = b;
        J->lo = m * t / nthreads; J->hi = m * (t + 1) / nthreads;
        started[t] = t > 0 && pthread_create(&th[t], NULL, run_cl, J) == 0;
    }
    run_cl(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) {
        if (started[t]) pthread_join(th[t], NULL);
        else run_cl(&jobs[t]);
    }
}
