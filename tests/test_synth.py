"""The input generators: the C twin of the R-MAT draws equals the numpy
definition draw for draw, and the generators are deterministic per seed."""
import numpy as np

import synth


def test_rmat_c_twin_equals_the_numpy_definition():
    assert synth._rmat_lib() is not None
    for n, ef, sb in [(1, 4, 0), (2, 3, 4), (1000, 16, 100), (3001, 16, 104), (65536, 8, 7)]:
        a = synth.rmat(n, ef, 3, plant_size=min(30, n), stream_base=sb)
        b = synth.rmat(n, ef, 3, plant_size=min(30, n), stream_base=sb, use_c=False)
        for x, y in zip(a[1:], b[1:]):
            assert np.array_equal(x, y), (n, ef, sb)


def test_chung_lu_c_twin_equals_the_numpy_definition():
    for n, md, seed in [(50, 4.0, 1), (3000, 12.0, 9), (100000, 20.0, 2)]:
        a = synth.chung_lu(n, md, 2.5, seed, plant_size=20, plant_prob=0.9)
        b = synth.chung_lu(n, md, 2.5, seed, plant_size=20, plant_prob=0.9, use_c=False)
        for x, y in zip(a[1:], b[1:]):
            assert np.array_equal(x, y), (n, md, seed)


def test_rmat_shape():
    n, s, d, planted = synth.rmat(5000, 16, 3, plant_size=30, plant_prob=1.0, stream_base=100)
    assert s.dtype == np.int32 and s.size == d.size >= 16 * 5000
    assert s.min() >= 0 and max(s.max(), d.max()) < n
    assert planted.size == 30 and np.all(np.diff(planted) > 0)
    # skew: the lowest ids carry most of the R-MAT mass (a = 0.57 quadrant)
    deg = np.bincount(np.concatenate([s, d]), minlength=n)
    assert deg[: n // 16].sum() > deg[-(n // 16):].sum() * 4


def test_generators_are_deterministic():
    a = synth.batch_rmat_graph(5, 1234)
    b = synth.batch_rmat_graph(5, 1234)
    assert all(np.array_equal(x, y) for x, y in zip(a[1:], b[1:]))
    c = synth.batch_rmat_graph(6, 1234)
    assert not np.array_equal(a[1], c[1])


def test_chung_lu_benchmark_graph_has_the_stated_shape():
    """The benchmark workload (Chung-Lu, n = 1e5, mean degree 20, degree
    exponent 2.5, a planted 60-node near-clique at edge probability 0.9,
    seed 2): the simple graph keeps a mean degree near 20 after duplicates
    and self-loops go, the planted nodes are adjacent with probability near
    0.9, and the degrees are heavy-tailed (the largest far above the mean)."""
    n, s, d, planted = synth.chung_lu(100_000, 20.0, 2.5, 2, plant_size=60, plant_prob=0.9)
    keep = s != d
    u, v = np.minimum(s[keep], d[keep]), np.maximum(s[keep], d[keep])
    key = np.unique(u.astype(np.int64) * n + v)
    m = key.size
    assert n == 100_000 and 19.0 < 2 * m / n < 21.0
    deg = np.bincount(np.concatenate([key // n, key % n]), minlength=n)
    assert deg.max() > 20 * 2 * m / n
    pset = np.zeros(n, bool)
    pset[planted] = True
    inside = np.count_nonzero(pset[key // n] & pset[key % n])
    assert planted.size == 60 and 0.85 < inside / (60 * 59 / 2) < 0.95


def test_batch_and_serving_recipes():
    """The batched workload's 256 instances: n log-uniform in [1e3, 1e5]
    (about half below the geometric midpoint 1e4) and k uniform in {3..8};
    the serving stream: exponential gaps of mean 1/200 s, k uniform in
    {3..10}, queries spread over the whole pool."""
    ns, ks = synth.batch_rmat_specs(256)
    assert ns.size == ks.size == 256 and ns.min() >= 1000 and ns.max() <= 100_000
    assert 100 < np.count_nonzero(ns < 10_000) < 156
    assert set(ks.tolist()) == set(range(3, 9))
    t, g, k = synth.serving_stream(4000, 200.0, 64)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() * 200.0 - 1.0) < 0.05
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.08     # exponential: cv = 1
    assert set(k.tolist()) == set(range(3, 11)) and set(g.tolist()) == set(range(64))


def test_er2000_has_the_expected_edges_and_triangles():
    """G(2000, 0.01) from seed 1: about C(2000, 2) p = 19,990 edges and
    C(2000, 3) p^3 = 1,331 triangles expected (each within a few standard
    deviations), counted by the oracle's explicit listing."""
    import oracle as O
    n, s, d = synth.workload_er2000()
    off, adj = O.csr(n, s, d)
    m = adj.size // 2
    assert n == 2000 and abs(m - 19_990) < 5 * np.sqrt(19_990)
    c3 = O.count_cliques(n, off, adj, 3)
    assert abs(c3 - 1331) < 6 * np.sqrt(1331)
