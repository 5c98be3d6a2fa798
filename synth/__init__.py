"""Seeded synthetic graph generators shared by the oracle tests, the CUDA
parity tests and the benchmark.

This module holds no arithmetic of the k-clique densest-subgraph method: it
only draws edge lists.  Every random number comes from SplitMix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
used as a counter-based generator:

    value(seed, i) = mix64(seed + (i + 1) * GAMMA),  GAMMA = 0x9E3779B97F4A7C15

where mix64 is the published SplitMix64 output finaliser.  Independent streams
of one seed use ``stream_seed(seed, s) = value(seed ^ STREAM_SALT, s)``.
Uniform doubles are ``(x >> 11) * 2**-53``.

The generators return *raw* draws as two int32 arrays (src, dst): they may
contain duplicate edges, both orientations of an edge and self-loops.  The
graph loader of the solver (and the oracle's own loader) symmetrises,
deduplicates and drops self-loops, so raw draws exercise that step.

The paper measures on SNAP/KONECT graphs (Table 3), which are not available
here; these generators stand in for them with the degree skew, mean degree and
dense planted regions of those workloads.
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
STREAM_SALT = 0xD1B54A32D192ED03
_TWO_M53 = float(2.0 ** -53)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64: output number ``index`` of the generator
    seeded with ``seed`` (index 0 is the first output)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx + np.uint64(1)) * GAMMA
    return _mix64(z)


def stream_seed(seed: int, stream: int) -> int:
    """Seed of independent stream ``stream`` derived from ``seed``."""
    v = splitmix64((seed ^ STREAM_SALT) & 0xFFFFFFFFFFFFFFFF,
                   np.array([stream], dtype=np.uint64))
    return int(v[0])


def uniforms(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """``count`` uniform doubles in [0, 1) from positions start..start+count-1
    of stream ``stream``."""
    s = stream_seed(seed, stream)
    x = splitmix64(s, np.arange(start, start + count, dtype=np.uint64))
    return (x >> np.uint64(11)).astype(np.float64) * _TWO_M53


def _as_edges(src, dst):
    return (np.ascontiguousarray(src, dtype=np.int32),
            np.ascontiguousarray(dst, dtype=np.int32))


# ---------------------------------------------------------------------------
# The paper's worked example G1 (7 nodes u0..u6, 9 triangles).
# The figure is not reproduced in the text, but the edge set is fixed by the
# five SCT pairs the paper prints for it (Example 2.2): every pair's V(P) is a
# clique, which yields these 13 edges, and no further edge can be added without
# creating a tenth triangle.
# ---------------------------------------------------------------------------
G1_EDGES = [(0, 1), (0, 3), (1, 3), (1, 2), (1, 6), (2, 3), (2, 6), (3, 6),
            (3, 4), (3, 5), (4, 5), (4, 6), (5, 6)]


def g1():
    """Return (n, src, dst) of the paper's example graph G1."""
    e = np.array(G1_EDGES, dtype=np.int32)
    return 7, *_as_edges(e[:, 0], e[:, 1])


def erdos_renyi(n: int, p: float, seed: int):
    """G(n, p): each unordered pair {i < j} (lexicographic pair index t) is an
    edge iff uniform(stream 0, t) < p."""
    iu, ju = np.triu_indices(n, k=1)
    u = uniforms(seed, 0, 0, iu.size)
    keep = u < p
    return n, *_as_edges(iu[keep], ju[keep])


def _plant(n: int, size: int, prob: float, seed: int, stream_pick: int,
           stream_edge: int):
    """Pick ``size`` distinct nodes uniformly (the ``size`` smallest random
    keys of stream ``stream_pick``) and add each pair among them with
    probability ``prob`` (stream ``stream_edge``, pair index in lexicographic
    order of the sorted node list)."""
    if size <= 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64)
    keys = uniforms(seed, stream_pick, 0, n)
    nodes = np.sort(np.argsort(keys, kind="stable")[:size]).astype(np.int64)
    ia, ja = np.triu_indices(size, k=1)
    u = uniforms(seed, stream_edge, 0, ia.size)
    keep = u < prob
    return nodes, nodes[ia[keep]], nodes[ja[keep]]


def chung_lu(n: int, mean_degree: float, beta: float, seed: int,
             plant_size: int = 0, plant_prob: float = 1.0, use_c: bool = True):
    """Chung-Lu power-law graph.

    Weights w_i = (i+1)^(-1/(beta-1)), scaled to mean ``mean_degree`` and
    clipped at sqrt(n * mean_degree).  ``round(n * mean_degree / 2)`` edge
    draws pick both endpoints independently with probability proportional to w
    (inverse-CDF sampling on the cumulative weights, streams 0 and 1).  A
    near-clique of ``plant_size`` uniformly chosen nodes with edge probability
    ``plant_prob`` is added (streams 2 and 3).
    Returns (n, src, dst, planted_nodes)."""
    i = np.arange(n, dtype=np.float64)
    w = (i + 1.0) ** (-1.0 / (beta - 1.0))
    w *= mean_degree / w.mean()
    w = np.minimum(w, np.sqrt(n * mean_degree))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m = int(round(n * mean_degree / 2.0))
    L = _rmat_lib() if use_c else None
    if L is None:
        ua = uniforms(seed, 0, 0, m)
        ub = uniforms(seed, 1, 0, m)
        a = np.minimum(np.searchsorted(cdf, ua, side="right"), n - 1)
        b = np.minimum(np.searchsorted(cdf, ub, side="right"), n - 1)
    else:   # the C twin of the three lines above
        import os
        cdf = np.ascontiguousarray(cdf, np.float64)
        a = np.empty(m, np.int64)
        b = np.empty(m, np.int64)
        L.synth_chunglu_draws(stream_seed(seed, 0), stream_seed(seed, 1), m, cdf.ctypes.data, n,
                              a.ctypes.data, b.ctypes.data, min(os.cpu_count() or 1, 64))
    nodes, pa, pb = _plant(n, plant_size, plant_prob, seed, 2, 3)
    src = np.concatenate([a, pa])
    dst = np.concatenate([b, pb])
    return n, *_as_edges(src, dst), nodes.astype(np.int32)


_clib = None


def _rmat_lib():
    """The C twin of ``_rmat_block_numpy`` (synth/_rmat.c, built with gcc on
    first use into synth/_build); None when it cannot be built."""
    global _clib
    if _clib is None:
        import ctypes as C
        import os
        import subprocess
        here = os.path.dirname(os.path.abspath(__file__))
        so = os.path.join(here, "_build", "librmat.so")
        srcf = os.path.join(here, "_rmat.c")
        try:
            if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(srcf):
                os.makedirs(os.path.dirname(so), exist_ok=True)
                tmp = so + f".{os.getpid()}.tmp"
                subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                                       srcf, "-o", tmp])
                os.replace(tmp, so)
            L = C.CDLL(so)
            L.synth_rmat_block.restype = C.c_int64
            L.synth_rmat_block.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_int, C.c_double,
                                           C.c_double, C.c_double, C.c_int64, C.c_void_p,
                                           C.c_void_p, C.c_int]
            L.synth_chunglu_draws.restype = None
            L.synth_chunglu_draws.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, C.c_void_p,
                                              C.c_int64, C.c_void_p, C.c_void_p, C.c_int]
            _clib = L
        except (OSError, subprocess.CalledProcessError):
            _clib = False
    return _clib or None


def _rmat_block_numpy(sseed_stream: tuple, base: int, cnt: int, scale: int, a, ab, abc, n):
    """One block of R-MAT draws (the definition): draw j takes the uniforms
    at positions base + j * scale + l, l < scale, of the stream; draws with an
    endpoint >= n are dropped."""
    seed, stream = sseed_stream
    u = uniforms(seed, stream, base, cnt * scale).reshape(cnt, scale)
    src = np.zeros(cnt, dtype=np.int64)
    dst = np.zeros(cnt, dtype=np.int64)
    for lvl in range(scale):
        x = u[:, lvl]
        bit = np.int64(1) << np.int64(scale - 1 - lvl)
        right = ((x >= a) & (x < ab)) | (x >= abc)
        down = x >= ab
        src += np.where(down, bit, 0)
        dst += np.where(right, bit, 0)
    ok = (src < n) & (dst < n)
    return src[ok], dst[ok]


def _rmat_block(seed, stream, base, cnt, scale, a, ab, abc, n, use_c=True):
    L = _rmat_lib() if use_c else None
    if L is None:
        return _rmat_block_numpy((seed, stream), base, cnt, scale, a, ab, abc, n)
    import os
    src = np.empty(cnt, np.int64)
    dst = np.empty(cnt, np.int64)
    kept = L.synth_rmat_block(stream_seed(seed, stream), base, cnt, scale, a, ab, abc, n,
                              src.ctypes.data, dst.ctypes.data, min(os.cpu_count() or 1, 64))
    return src[:kept], dst[:kept]


def rmat(n: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19,
         plant_size: int = 0, plant_prob: float = 1.0, stream_base: int = 0,
         use_c: bool = True):
    """R-MAT graph on n nodes (scale = ceil(log2 n)) with ``edge_factor * n``
    edge draws.  Each draw descends ``scale`` levels choosing quadrant
    (a, b, c, d = 1-a-b-c) from one uniform per level; draws with an endpoint
    >= n are redrawn from the next attempt block of the same stream.  A
    near-clique of ``plant_size`` nodes (probability ``plant_prob``) is added.
    Returns (n, src, dst, planted_nodes)."""
    scale = max(1, int(np.ceil(np.log2(max(n, 2)))))
    want = edge_factor * n
    out_s, out_d = [], []
    have = 0
    attempt = 0
    ab, abc = a + b, a + b + c
    while have < want:
        cnt = int((want - have) * 1.1) + 16
        src, dst = _rmat_block(seed, stream_base + 0, attempt * (1 << 40), cnt, scale, a, ab,
                               abc, n, use_c)
        take = min(src.size, want - have)
        out_s.append(src[:take])
        out_d.append(dst[:take])
        have += take
        attempt += 1
    nodes, pa, pb = _plant(n, plant_size, plant_prob, seed, stream_base + 2,
                           stream_base + 3)
    src = np.concatenate(out_s + [pa])
    dst = np.concatenate(out_d + [pb])
    return n, *_as_edges(src, dst), nodes.astype(np.int32)


def random_small(n: int, p: float, seed: int):
    """Small G(n, p) graphs for brute-force checks (n <= 20)."""
    return erdos_renyi(n, p, seed)


# ---------------------------------------------------------------------------
# Workload recipes (the graphs the tests and the benchmark use).
# ---------------------------------------------------------------------------

def workload_er2000():
    """Erdos-Renyi G(2000, 0.01), seed 1 (k = 3, T = 100)."""
    return erdos_renyi(2000, 0.01, 1)


def workload_chunglu_1e5():
    """Chung-Lu n = 1e5, mean degree 20, exponent 2.5, planted 60-node
    near-clique at edge probability 0.9, seed 2 (k = 5, T = 200)."""
    n, s, d, _ = chung_lu(100_000, 20.0, 2.5, 2, plant_size=60, plant_prob=0.9)
    return n, s, d


def workload_rmat24():
    """The large single graph: R-MAT scale 24 (16,777,216 nodes), edge factor
    32 (536,870,912 draws), planted 200-node near-clique at p = 0.95, seed 4."""
    n, s, d, _ = rmat(1 << 24, 32, 4, plant_size=200, plant_prob=0.95)
    return n, s, d


def batch_rmat_specs(count: int = 256, seed: int = 3, nmin=1e3, nmax=1e5):
    """Per-instance (n, k) of the batched workload: n log-uniform in
    [nmin, nmax], k uniform in {3..8}; stream 10 and 11 of ``seed``."""
    un = uniforms(seed, 10, 0, count)
    uk = uniforms(seed, 11, 0, count)
    ns = np.rint(np.exp(np.log(nmin) + un * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    ks = 3 + np.minimum((uk * 6).astype(np.int64), 5)
    return ns, ks


def batch_rmat_graph(i: int, n: int, seed: int = 3):
    """Instance ``i`` of the batched workload: R-MAT edge factor 16 with a
    planted 30-node clique; streams 100 + 4 i ... of ``seed``."""
    n, s, d, _ = rmat(int(n), 16, seed, plant_size=30, plant_prob=1.0,
                      stream_base=100 + 4 * i)
    return n, s, d


def serving_pool(count: int = 32, seed: int = 5, nmin=1e3, nmax=1e6):
    """Graphs of the serving workload: the Chung-Lu generator of the n = 1e5
    workload (mean degree 20, exponent 2.5, planted 60-node near-clique at
    p = 0.9) with n log-uniform in [nmin, nmax] (stream 20 of ``seed``);
    graph i draws from seed * 1000 + i."""
    un = uniforms(seed, 20, 0, count)
    ns = np.rint(np.exp(np.log(nmin) + un * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    out = []
    for i, n in enumerate(ns):
        n, s, d, _ = chung_lu(int(n), 20.0, 2.5, seed * 1000 + i, plant_size=60, plant_prob=0.9)
        out.append((n, s, d))
    return out


def serving_stream(count: int, rate: float, pool_size: int, seed: int = 5):
    """Arrival times (s) of a Poisson stream of ``rate`` queries/s
    (exponential gaps, stream 21), the pool graph of each query (stream 22)
    and its k, uniform in {3..10} (stream 23)."""
    gaps = -np.log1p(-uniforms(seed, 21, 0, count)) / rate
    g = np.minimum((uniforms(seed, 22, 0, count) * pool_size).astype(np.int64), pool_size - 1)
    k = 3 + np.minimum((uniforms(seed, 23, 0, count) * 8).astype(np.int64), 7)
    return np.cumsum(gaps), g, k
