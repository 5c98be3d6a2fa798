"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results -- CSR, core numbers, peel rounds, vertex order, the SCT in
canonical form, c_k, the rule-I ranking r_T and the extracted prefix -- are
compared bit for bit.  The FP32 continuous path is compared with the oracle's
FP64 continuous rule within 1e-5 relative (infinity norm) for one iteration
from the same state at every horizon and for short horizons from zero; at
full horizons it must keep Lemma 3.1's invariants and extract a density
within 1% of the oracle's.
"""
import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K
import synth
from conftest import load_golden

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)


def gpu_pairs(sct):
    p = K.kdss_sct_copy_pairs(sct)
    po, nodes, h = p["pair_off"], p["nodes"], p["h"]
    out = []
    for q in range(len(h)):
        seg = nodes[po[q]:po[q + 1]]
        assert np.all(np.diff(seg & 0x7FFFFFFF) > 0), "pair nodes not ascending by id"
        hold = tuple(int(x) & 0x7FFFFFFF for x in seg if x < 0)
        piv = tuple(int(x) for x in seg if x >= 0)
        assert len(hold) == h[q]
        out.append((hold, piv))
    return sorted(out)


def oracle_graph(n, s, d, k, kind):
    off, adj = O.csr(n, s, d)
    core, rnd, dg = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd, kind)
    sc = O.sct(n, off, adj, rank, vert, k)
    return dict(off=off, adj=adj, core=core, round=rnd, rank=rank, vert=vert, sct=sc, degen=dg)


def oracle_extract(n, sc, k, r, T):
    order = O.sort_desc(r)
    lo, hi, flo, fhi = O.prefix_counts_pairs(n, order, sc, k)
    i = O.argmax_density(lo, hi)
    F = [int(a) | (int(b) << 64) for a, b in zip(flo, fhi)]
    return dict(istar=i, ids=np.sort(order[:i]), count=int(lo[i]) | (int(hi[i]) << 64),
                rho_prime=max(F[j] / j for j in range(1, n + 1)),
                upper_bound=float(np.max(r)) / T)


GRAPHS = {
    "g1": lambda: synth.g1(),
    "er300": lambda: synth.erdos_renyi(300, 0.08, 5),
    "chunglu3k": lambda: synth.chung_lu(3000, 12.0, 2.4, 9, plant_size=25, plant_prob=0.85)[:3],
    "rmat2k": lambda: synth.rmat(2000, 12, 11, plant_size=20, plant_prob=0.95)[:3],
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("kind", [K.KDSS_ORDER_PEEL, K.KDSS_ORDER_CORE])
def test_graph_build_matches_oracle(name, kind):
    n, s, d = GRAPHS[name]()
    sct = K.kdss_build_sct(n, s, d, 3, K.make_opts(order=kind, flags=K.KDSS_FLAG_KEEP_GRAPH))
    g = K.kdss_sct_copy_graph(sct)
    o = oracle_graph(n, s, d, 3, kind)
    assert np.array_equal(g["off"], o["off"]) and np.array_equal(g["adj"], o["adj"])
    assert np.array_equal(g["core"], o["core"])
    assert np.array_equal(g["round"], o["round"])
    assert np.array_equal(g["rank"], o["rank"])
    assert K.kdss_sct_info(sct)["degeneracy"] == o["degen"]


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [2, 3, 4, 6])
@pytest.mark.parametrize("kind", [K.KDSS_ORDER_PEEL, K.KDSS_ORDER_CORE])
def test_sct_matches_oracle(name, k, kind):
    n, s, d = GRAPHS[name]()
    sct = K.kdss_build_sct(n, s, d, k, K.make_opts(order=kind))
    o = oracle_graph(n, s, d, k, kind)
    info = K.kdss_sct_info(sct)
    assert info["eta_k"] == len(o["sct"]["h"])
    assert info["L_k"] == len(o["sct"]["nodes"])
    assert gpu_pairs(sct) == O.canonical_pairs(o["sct"])
    ck = sum(O.binom(int(o["sct"]["pair_off"][q + 1] - o["sct"]["pair_off"][q]) - int(hq), k - int(hq))
             for q, hq in enumerate(o["sct"]["h"]))
    assert info["c_k"] == ck


def test_g1_example_2_2_on_the_gpu():
    G = load_golden("g1_example.txt")
    n, s, d = synth.g1()
    sct = K.kdss_build_sct(n, s, d, 3, K.make_opts(order=K.KDSS_ORDER_CORE))
    want = []
    for ln in G["pair"]:
        a, b = ln.split("|")
        want.append((tuple(sorted(map(int, a.split()))), tuple(sorted(map(int, b.split())))))
    assert gpu_pairs(sct) == sorted(want)
    assert K.kdss_sct_info(sct)["c_k"] == int(G["triangles"][0])
    res = K.kdss_solve(n, s, d, 3, 100)
    assert res["istar"] == 6 and res["ids"].tolist() == [1, 2, 3, 4, 5, 6] and res["count"] == 8


@pytest.mark.parametrize("prec", [K.KDSS_INT64, K.KDSS_FP64])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_fw_on_the_oracle_sct_is_bit_exact(name, prec):
    """The PBUpdate kernels fed the oracle's own SCT reproduce r_T exactly."""
    n, s, d = GRAPHS[name]()
    k, T = 4, 37
    o = oracle_graph(n, s, d, k, K.KDSS_ORDER_PEEL)
    sc = o["sct"]
    sct = K.kdss_sct_from_pairs(n, k, sc["pair_off"], sc["nodes"], sc["h"])
    st = K.kdss_fw_iterate(sct, None, T, K.make_opts(precision=prec))
    r, t = K.kdss_state_copy_r(st, n, prec)
    assert t == T
    want = O.fw_sync(n, sc, k, T)
    assert np.array_equal(r.astype(np.uint64), want)


def _random_pairs(n, npairs, k, maxlen, seed):
    rng = np.random.default_rng(seed)
    po, nodes, hs = [0], [], []
    for _ in range(npairs):
        ln = int(rng.integers(k, maxlen + 1))
        h = int(rng.integers(0, min(k, ln) + 1))
        ids = rng.choice(n, size=ln, replace=False)
        nodes.extend(ids.tolist())
        hs.append(h)
        po.append(len(nodes))
    return dict(pair_off=np.array(po, np.int64), nodes=np.array(nodes, np.int32),
                h=np.array(hs, np.int32))


@pytest.mark.parametrize("maxlen", [8, 16, 32, 256, 700])
def test_fw_every_length_class_is_bit_exact(maxlen):
    """Pairs of every length class (and ragged lengths inside each) through
    kdss_sct_from_pairs; h ranges over 0..k, so zero-cap pivots occur."""
    n, k, T = 900, 4, 9
    sc = _random_pairs(n, 300 if maxlen <= 256 else 40, k, maxlen, maxlen)
    sct = K.kdss_sct_from_pairs(n, k, sc["pair_off"], sc["nodes"], sc["h"])
    st = K.kdss_fw_iterate(sct, None, T, K.make_opts())
    r, _ = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
    assert np.array_equal(r, O.fw_sync(n, sc, k, T))
    res = K.kdss_extract(sct, st)
    want = oracle_extract(n, sc, k, r, T)
    assert res["istar"] == want["istar"] and res["count"] == want["count"]
    assert res["ids"].tolist() == want["ids"].tolist()


def _many_short_pairs(n, npairs, k, seed):
    """npairs pairs of k..32 distinct nodes of [0, n), n prime: pair q is the
    progression a_q + j b_q (mod n), j < len_q, with b_q != 0."""
    rng = np.random.default_rng(seed)
    ln = rng.integers(k, 33, size=npairs)
    a = np.repeat(rng.integers(0, n, size=npairs), ln)
    b = np.repeat(rng.integers(1, n, size=npairs), ln)
    po = np.zeros(npairs + 1, np.int64)
    po[1:] = np.cumsum(ln)
    j = np.arange(po[-1]) - np.repeat(po[:-1], ln)
    nodes = ((a + j * b) % n).astype(np.int32)
    h = rng.integers(0, k + 1, size=npairs).astype(np.int32)
    return dict(pair_off=po, nodes=nodes, h=h)


def test_fw_pipelined_slow_walk_is_bit_exact():
    """With at least 64 short pairs per warp of the slow kernels' grid (152
    SMs x 8 blocks x 8 warps) the slow kernels pipeline their loads across
    pairs: r_T bit-exact for INT64 and FP64, the FP32 rule within 1e-5 of the
    FP64 continuous oracle over a short horizon."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n, k, T = 20011, 4, 6
    sc = _many_short_pairs(n, 64 * 8 * 8 * sms + 12345, k, 5)
    sct = K.kdss_sct_from_pairs(n, k, sc["pair_off"], sc["nodes"], sc["h"])
    want = O.fw_sync_par(n, sc, k, T)
    for prec in (K.KDSS_INT64, K.KDSS_FP64):
        st = K.kdss_fw_iterate(sct, None, T, K.make_opts(precision=prec))
        r, _ = K.kdss_state_copy_r(st, n, prec)
        assert np.array_equal(r.astype(np.uint64), want)
    T32 = 3
    r32, _ = K.kdss_state_copy_r(_fp32_state(sct, T32), n, K.KDSS_FP32K)
    r64 = O.fw_cont(n, sc, k, T32) / T32
    err = np.max(np.abs(r32.astype(np.float64) - r64)) / max(np.max(np.abs(r64)), 1e-300)
    assert err <= FP32_RTOL, err


def test_fw_large_counts_are_bit_exact():
    """Pairs of 24-32 nodes sharing a hub with k = 14: per-pair counts up to
    C(31, 13) ~ 2e8 push r beyond 2^32 within the run (64-bit arithmetic in
    the fast first step and in the full walk)."""
    rng = np.random.default_rng(21)
    n, k, T = 400, 14, 20
    po, nodes, hs = [0], [], []
    for _ in range(2500):
        ln = int(rng.integers(24, 33))
        ids = [0] + rng.choice(np.arange(1, n), size=ln - 1, replace=False).tolist()
        h = int(rng.integers(1, 4))
        nodes.extend(ids)
        hs.append(h)
        po.append(len(nodes))
    sc = dict(pair_off=np.array(po, np.int64), nodes=np.array(nodes, np.int32),
              h=np.array(hs, np.int32))
    sct = K.kdss_sct_from_pairs(n, k, sc["pair_off"], sc["nodes"], sc["h"])
    want = O.fw_sync(n, sc, k, T)
    assert int(want.max()) > (1 << 32)
    for prec in (K.KDSS_INT64, K.KDSS_FP64):
        st = K.kdss_fw_iterate(sct, None, T, K.make_opts(precision=prec))
        r, _ = K.kdss_state_copy_r(st, n, prec)
        assert np.array_equal(r.astype(np.uint64), want)


def test_profiled_and_graph_runs_agree():
    """The profiled per-iteration path (every 8th iteration as separate graphs
    between events, the others fused) and the default path (the resident
    launch) give the same r for the integer rule.  For the continuous FP32
    rule the two forms add their allocations in different orders, and the
    rule's trajectory amplifies rounding differences (a 1e-13 perturbation
    grows about 100x per 10 iterations), so after 30 iterations they agree in
    what the iterations fix -- sum r-hat = c_k -- and in the extracted
    density; per-iteration agreement with the FP64 oracle is tested in
    test_fp32_one_iteration_matches_fp64_oracle."""
    n, s, d = GRAPHS["rmat2k"]()
    sct = K.kdss_build_sct(n, s, d, 4)
    ck = K.kdss_sct_info(sct)["c_k"]
    for prec in (K.KDSS_INT64, K.KDSS_FP64, K.KDSS_FP32K):
        a = K.kdss_fw_iterate(sct, None, 30, K.make_opts(
            precision=prec, flags=K.KDSS_FLAG_PROFILE | K.KDSS_FLAG_PER_ITERATION))
        b = K.kdss_fw_iterate(sct, None, 30, K.make_opts(precision=prec))
        ra, _ = K.kdss_state_copy_r(a, n, prec)
        rb, _ = K.kdss_state_copy_r(b, n, prec)
        if prec == K.KDSS_FP32K:
            for r in (ra, rb):
                assert abs(float(r.astype(np.float64).sum()) - ck) <= FP32_RTOL * ck
            da, db = K.kdss_extract(sct, a)["density"], K.kdss_extract(sct, b)["density"]
            assert abs(da - db) <= 0.01 * db
        else:
            assert np.array_equal(ra, rb)
        tm = K.kdss_state_timing(a)
        assert tm["fw_launches"] == 4 and tm["fw_kernel_ms"] > 0   # iterations 0, 8, 16, 24


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [3, 5])
def test_whole_path_matches_oracle(name, k):
    n, s, d = GRAPHS[name]()
    T = 60
    o = oracle_graph(n, s, d, k, K.KDSS_ORDER_PEEL)
    sct = K.kdss_build_sct(n, s, d, k)
    st = K.kdss_fw_iterate(sct, None, T)
    r, _ = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
    ro = O.fw_sync(n, o["sct"], k, T)
    assert np.array_equal(r, ro)
    res = K.kdss_extract(sct, st)
    want = oracle_extract(n, o["sct"], k, ro, T) if n else None
    if len(o["sct"]["h"]) == 0:
        return
    assert res["istar"] == want["istar"]
    assert res["ids"].tolist() == want["ids"].tolist()
    assert res["count"] == want["count"]
    assert abs(res["rho_prime"] - want["rho_prime"]) <= 1e-12 * max(1.0, want["rho_prime"])
    assert abs(res["upper_bound"] - want["upper_bound"]) <= 1e-12 * max(1.0, want["upper_bound"])
    assert res["rho_prime"] <= res["upper_bound"] * (1 + 1e-12)   # weak duality (Thm 3.5-3.6)


def test_resume_equals_uninterrupted_run():
    n, s, d = GRAPHS["chunglu3k"]()
    sct = K.kdss_build_sct(n, s, d, 4)
    a = K.kdss_fw_iterate(sct, None, 25)
    a = K.kdss_fw_iterate(sct, a, 15)
    b = K.kdss_fw_iterate(sct, None, 40)
    ra, ta = K.kdss_state_copy_r(a, n, K.KDSS_INT64)
    rb, tb = K.kdss_state_copy_r(b, n, K.KDSS_INT64)
    assert ta == tb == 40 and np.array_equal(ra, rb)


def _fp32_state(sct, T, flags=0):
    return (K.kdss_fw_iterate(sct, None, T, K.make_opts(precision=K.KDSS_FP32K, flags=flags))
            if T > 0 else None)


@pytest.mark.parametrize("name", ["er300", "chunglu3k", "rmat2k"])
@pytest.mark.parametrize("t", [1, 2, 5, 30, 80])
@pytest.mark.parametrize("flags", [0, K.KDSS_FLAG_PER_ITERATION])
def test_fp32_one_iteration_matches_fp64_oracle(name, t, flags):
    """From the GPU's own r_{t-1}/(t-1), one FP32 iteration of the continuous
    rule equals one FP64 oracle iteration within 1e-5 (relative, inf-norm),
    in the resident launch (default) and in the per-iteration kernels.
    Over many iterations the continuous rule amplifies rounding differences
    (a 1e-13 perturbation grows about 100x per 10 iterations), so agreement is
    checked per iteration, at every horizon."""
    n, s, d = GRAPHS[name]()
    k = 4
    o = oracle_graph(n, s, d, k, K.KDSS_ORDER_PEEL)
    sct = K.kdss_build_sct(n, s, d, k)
    st = _fp32_state(sct, t - 1, flags)
    prev = K.kdss_state_copy_r(st, n, K.KDSS_FP32K)[0].astype(np.float64) if st else np.zeros(n)
    st = K.kdss_fw_iterate(sct, st, 1, K.make_opts(precision=K.KDSS_FP32K, flags=flags))
    got, tt = K.kdss_state_copy_r(st, n, K.KDSS_FP32K)
    assert tt == t
    want = O.fw_cont(n, o["sct"], k, 1, r0=prev * (t - 1)) / t
    err = np.max(np.abs(got.astype(np.float64) - want)) / max(np.max(np.abs(want)), 1e-300)
    assert err <= FP32_RTOL, err


@pytest.mark.parametrize("name", ["er300", "chunglu3k", "rmat2k"])
def test_fp32_short_horizon_from_zero(name):
    n, s, d = GRAPHS[name]()
    k, T = 4, 4
    o = oracle_graph(n, s, d, k, K.KDSS_ORDER_PEEL)
    sct = K.kdss_build_sct(n, s, d, k)
    r32, _ = K.kdss_state_copy_r(_fp32_state(sct, T), n, K.KDSS_FP32K)
    r64 = O.fw_cont(n, o["sct"], k, T) / T
    err = np.max(np.abs(r32.astype(np.float64) - r64)) / max(np.max(np.abs(r64)), 1e-300)
    assert err <= FP32_RTOL, err


def _check_fp32_invariants(n, s, d, k, T, sct, st, o):
    r32, _ = K.kdss_state_copy_r(st, n, K.KDSS_FP32K)
    ck = K.kdss_sct_info(sct)["c_k"]
    # Lemma 3.1: sum_u r(u) = |C_k(V)|, r(u) <= #k-cliques containing u
    assert abs(float(r32.astype(np.float64).sum()) - ck) <= FP32_RTOL * ck
    cnt = np.zeros(n)
    sc = o["sct"]
    for q in range(len(sc["h"])):
        seg = sc["nodes"][sc["pair_off"][q]:sc["pair_off"][q + 1]]
        h = int(sc["h"][q]); p = len(seg) - h
        cnt[seg[:h]] += O.binom(p, k - h)
        if k - h - 1 >= 0 and p >= 1:
            cnt[seg[h:]] += O.binom(p - 1, k - h - 1)
    assert np.all(r32 <= cnt * (1 + FP32_RTOL) + 1e-6)
    res = K.kdss_extract(sct, st)
    want = oracle_extract(n, sc, k, O.fw_sync(n, sc, k, T), T)
    assert res["density"] >= 0.99 * want["count"] / want["istar"]
    assert res["rho_prime"] <= res["upper_bound"] * (1 + FP32_RTOL)   # weak duality
    return res


@pytest.mark.parametrize("name", ["er300", "chunglu3k", "rmat2k"])
def test_fp32_invariants_and_density_at_T80(name):
    n, s, d = GRAPHS[name]()
    k, T = 4, 80
    o = oracle_graph(n, s, d, k, K.KDSS_ORDER_PEEL)
    sct = K.kdss_build_sct(n, s, d, k)
    _check_fp32_invariants(n, s, d, k, T, sct, _fp32_state(sct, T), o)


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def test_empty_and_degenerate_inputs():
    # no nodes
    sct = K.kdss_build_sct(0, np.zeros(0, np.int32), np.zeros(0, np.int32), 3)
    assert K.kdss_sct_info(sct)["eta_k"] == 0
    res = K.kdss_solve(0, np.zeros(0, np.int32), np.zeros(0, np.int32), 3, 5)
    assert res["istar"] == 0
    # nodes but no edges; only self-loops and duplicates
    res = K.kdss_solve(10, np.array([3, 3, 4], np.int32), np.array([3, 3, 4], np.int32), 3, 5)
    assert res["count"] == 0
    # a graph with no k-clique
    n, s, d = synth.erdos_renyi(50, 0.02, 3)
    sct = K.kdss_build_sct(n, s, d, 6)
    assert K.kdss_sct_info(sct)["eta_k"] == 0
    st = K.kdss_fw_iterate(sct, None, 3)
    r, _ = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
    assert not r.any()
    # T = 0
    n, s, d = synth.g1()
    sct = K.kdss_build_sct(n, s, d, 3)
    st = K.kdss_fw_iterate(sct, None, 0)
    assert K.kdss_state_copy_r(st, n, K.KDSS_INT64)[1] == 0


def test_k_equal_clique_size_and_duplicate_heavy_input():
    # a 7-clique given with every edge three times in both orientations
    e = [(a, b) for a in range(7) for b in range(7) if a != b] * 3
    s = np.array([a for a, _ in e], np.int32)
    d = np.array([b for _, b in e], np.int32)
    res = K.kdss_solve(7, s, d, 7, 10)
    assert res["istar"] == 7 and res["count"] == 1
    res = K.kdss_solve(7, s, d, 2, 10)
    assert res["istar"] == 7 and res["count"] == 21


def test_errors_are_reported_not_crashed():
    with pytest.raises(K.KdssError) as e:
        K.kdss_build_sct(5, np.array([0, 7], np.int32), np.array([1, 2], np.int32), 3)
    assert e.value.code == K.KDSS_ERR_BAD_GRAPH
    with pytest.raises(K.KdssError) as e:
        K.kdss_build_sct(5, np.array([0], np.int32), np.array([1], np.int32), 1)
    assert e.value.code == K.KDSS_ERR_INVALID_ARG
    with pytest.raises(K.KdssError) as e:
        K.kdss_sct_from_pairs(5, 3, np.array([0, 2], np.int64), np.array([0, 1], np.int32),
                              np.array([1], np.int32))
    assert e.value.code == K.KDSS_ERR_INVALID_ARG   # |V(P)| = 2 < k
    # the library stays usable after errors
    n, s, d = synth.g1()
    assert K.kdss_solve(n, s, d, 3, 10)["istar"] == 6


def test_device_resident_input_and_torch_stream():
    import torch
    n, s, d = GRAPHS["chunglu3k"]()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        ts = torch.from_numpy(s).cuda()
        td = torch.from_numpy(d).cuda()
        a = K.kdss_solve(n, ts, td, 4, 30, K.make_opts(stream=st))
    b = K.kdss_solve(n, s, d, 4, 30, K.make_opts(allocator="library"))
    assert a["istar"] == b["istar"] and a["ids"].tolist() == b["ids"].tolist()
    assert a["count"] == b["count"]


# ---------------------------------------------------------------------------
# The two benchmark workloads at full size
# ---------------------------------------------------------------------------

def test_erdos_renyi_2000_k3_T100_full():
    n, s, d = synth.workload_er2000()
    k, T = 3, 100
    o = oracle_graph(n, s, d, k, K.KDSS_ORDER_PEEL)
    sct = K.kdss_build_sct(n, s, d, k)
    assert gpu_pairs(sct) == O.canonical_pairs(o["sct"])
    for prec in (K.KDSS_INT64, K.KDSS_FP64):
        st = K.kdss_fw_iterate(sct, None, T, K.make_opts(precision=prec))
        r, _ = K.kdss_state_copy_r(st, n, prec)
        ro = O.fw_sync(n, o["sct"], k, T)
        assert np.array_equal(r.astype(np.uint64), ro)
        res = K.kdss_extract(sct, st)
        want = oracle_extract(n, o["sct"], k, ro, T)
        assert (res["istar"], res["count"], res["ids"].tolist()) == \
            (want["istar"], want["count"], want["ids"].tolist())


def test_chung_lu_1e5_k5_T200_full():
    """The benchmark workload at full size, in the benchmark's launch
    configuration: canonical SCT, c_k, r_T (FP64 plain, bit-exact) and the
    extracted prefix against the oracle; the FP32 path's last iteration
    against the FP64 continuous oracle within 1e-5, its invariants and its
    density within 1%."""
    n, s, d = synth.workload_chunglu_1e5()
    k, T = 5, 200
    o = oracle_graph(n, s, d, k, K.KDSS_ORDER_PEEL)
    sct = K.kdss_build_sct(n, s, d, k)
    info = K.kdss_sct_info(sct)
    assert info["eta_k"] == len(o["sct"]["h"]) and info["L_k"] == len(o["sct"]["nodes"])
    assert gpu_pairs(sct) == O.canonical_pairs(o["sct"])
    st = K.kdss_fw_iterate(sct, None, T, K.make_opts(precision=K.KDSS_FP64))
    r, _ = K.kdss_state_copy_r(st, n, K.KDSS_FP64)
    ro = O.fw_sync(n, o["sct"], k, T)
    assert np.array_equal(r.astype(np.uint64), ro)
    assert int(ro.astype(object).sum()) == T * info["c_k"]
    res = K.kdss_extract(sct, st)
    want = oracle_extract(n, o["sct"], k, ro, T)
    assert (res["istar"], res["count"]) == (want["istar"], want["count"])
    assert res["ids"].tolist() == want["ids"].tolist()
    st32 = K.kdss_fw_iterate(sct, None, T - 1, K.make_opts(precision=K.KDSS_FP32K))
    prev = K.kdss_state_copy_r(st32, n, K.KDSS_FP32K)[0].astype(np.float64)
    st32 = K.kdss_fw_iterate(sct, st32, 1, K.make_opts(precision=K.KDSS_FP32K))
    got = K.kdss_state_copy_r(st32, n, K.KDSS_FP32K)[0].astype(np.float64)
    want1 = O.fw_cont(n, o["sct"], k, 1, r0=prev * (T - 1)) / T
    assert np.max(np.abs(got - want1)) / np.max(want1) <= FP32_RTOL
    _check_fp32_invariants(n, s, d, k, T, sct, st32, o)
