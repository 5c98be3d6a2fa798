"""The work-queue PBUpdate kernels (integer rule): the first step and the walk
of the pairs it leaves in one warp from the staged tile, longer pairs by
groups of 8 or 32 lanes, items taken from a device counter.  r_T must equal
the oracle's bit for bit for every item size and lanes-per-pair choice, on
graphs whose SCTs hold short pairs, pairs of 33..256 nodes and pairs of more
than 256 nodes; batches through the queue must equal kdss_solve per query and
report what the autotuner tried.
"""
import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)


def _planted(n, size, seed, p=0.95):
    n, s, d, _ = synth.chung_lu(n, 10.0, 2.4, seed, plant_size=size, plant_prob=p)
    return n, s, d


GRAPHS = {
    "chunglu3k": lambda: synth.chung_lu(3000, 12.0, 2.4, 31, plant_size=25, plant_prob=0.85)[:3],
    "long80": lambda: _planted(2500, 80, 32),          # pairs of 33..256 nodes
    "long300": lambda: _planted(1500, 300, 33, 1.0),   # pairs of more than 256 nodes
    "rmat2k": lambda: synth.rmat(2048, 16, 34, plant_size=20, plant_prob=1.0)[:3],
}


def _oracle_r(n, s, d, k, T):
    off, adj = O.csr(n, s, d)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    return O.fw_sync(n, O.sct(n, off, adj, rank, vert, k), k, T)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_queue_iterations_equal_the_oracle(name):
    n, s, d = GRAPHS[name]()
    k, T = 4, 12
    want = _oracle_r(n, s, d, k, T)
    sct = K.kdss_build_sct(n, s, d, k)
    cls = K.kdss_sct_info(sct)["pairs_per_class"]
    if name == "long80":
        assert cls[3] > 0
    if name == "long300":
        assert cls[4] > 0
    for chunk in (1, 4, 16):
        for tpp in (8, 32):
            for prec in (K.KDSS_INT64, K.KDSS_FP64):
                o = K.make_opts(precision=prec, chunk=chunk, threads_per_path=tpp)
                st = K.kdss_fw_iterate(sct, None, T, o)
                r, t = K.kdss_state_copy_r(st, n, prec)
                assert t == T
                assert np.array_equal(r.astype(np.uint64), want), (chunk, tpp, prec)


def test_queue_iterations_at_k_on_a_k_agnostic_sct():
    n, s, d = GRAPHS["long80"]()
    multi = K.kdss_build_sct_multi(n, s, d, 6)
    for k in (3, 5):
        st = K.kdss_fw_iterate_at(multi, k, None, 10, K.make_opts(chunk=4))
        r, _ = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
        assert np.array_equal(r, _oracle_r(n, s, d, k, 10))


def test_batch_through_the_queue_equals_solve_and_reports_tuning():
    qs = []
    for i, nn in enumerate([800, 1500, 2500, 1200]):
        n, s, d = synth.batch_rmat_graph(i, nn)
        qs.append((n, s, d, 3 + i, 30))
    qs.append((*GRAPHS["long80"](), 5, 30))
    out = K.kdss_solve_batch(qs, K.make_opts(precision=K.KDSS_INT64))
    tune = K.kdss_batch_last_tuning()
    assert tune["autotuned"] and len(tune["tried"]) >= 3
    assert (tune["chunk"], tune["threads_per_path"]) in \
        [(t["chunk"], t["threads_per_path"]) for t in tune["tried"]]
    for q, res in zip(qs, out):
        one = K.kdss_solve(*q)
        assert res["status"] == 0
        assert (res["istar"], res["count"], res["ids"].tolist()) == \
            (one["istar"], one["count"], one["ids"].tolist())
        assert res["upper_bound"] == one["upper_bound"]
    fixed = K.kdss_solve_batch(qs, K.make_opts(precision=K.KDSS_FP64, chunk=2,
                                               threads_per_path=8))
    t2 = K.kdss_batch_last_tuning()
    assert (t2["chunk"], t2["threads_per_path"], t2["autotuned"]) == (2, 8, False)
    for a, b in zip(out, fixed):
        assert (a["istar"], a["count"]) == (b["istar"], b["count"])


@pytest.mark.parametrize("name", ["chunglu3k", "long80", "long300"])
def test_fp32_queue_iterations_match_the_fp64_oracle(name):
    """The continuous rule on the work queue: one iteration from zero and four
    iterations agree with the FP64 oracle within 1e-5 (relative, inf-norm),
    for every item size and lanes-per-pair choice."""
    n, s, d = GRAPHS[name]()
    k = 4
    off, adj = O.csr(n, s, d)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    sc = O.sct(n, off, adj, rank, vert, k)
    sct = K.kdss_build_sct(n, s, d, k)
    for T in (1, 4):
        want = O.fw_cont(n, sc, k, T) / T
        for chunk, tpp in ((1, 32), (4, 8), (16, 32)):
            o = K.make_opts(precision=K.KDSS_FP32K, chunk=chunk, threads_per_path=tpp)
            got, t = K.kdss_state_copy_r(K.kdss_fw_iterate(sct, None, T, o), n, K.KDSS_FP32K)
            assert t == T
            err = np.max(np.abs(got.astype(np.float64) - want)) / np.max(np.abs(want))
            assert err <= 1e-5, (T, chunk, tpp, err)


def test_fp32_batch_through_the_queue_matches_the_oracle_density():
    qs = [(*synth.batch_rmat_graph(i, nn), 3 + i, 40) for i, nn in enumerate([900, 1700, 2600])]
    out = K.kdss_solve_batch(qs, K.make_opts(precision=K.KDSS_FP32K))
    assert K.kdss_batch_last_tuning()["autotuned"]
    for q, res in zip(qs, out):
        want = O.solve(*q)
        assert res["status"] == 0
        assert abs(res["density"] - want["density"]) <= 0.01 * want["density"]
