"""The resident launch of the integer-rule iterations: all T iterations of
Alg. 2 in one cooperative launch, the pair stream held in the blocks' shared
memory, r in two copies and the per-iteration delta in three vectors so that
each iteration ends on one grid barrier.

r_T must equal the oracle's synchronous iterations (Alg. 2 with Alg. 3, every
pair reading r_{t-1}) bit for bit, and the per-iteration launches
(KDSS_FLAG_PER_ITERATION) bit for bit, for INT64 and FP64, for runs split
over several calls, at a chosen k of a k-agnostic SCT, and through the
extraction (the bound max_u r(u)/t reads the running max the launch keeps).
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


GRAPHS = {
    "g1": lambda: synth.g1(),
    "er300": lambda: synth.erdos_renyi(300, 0.08, 51),
    "chunglu3k": lambda: synth.chung_lu(3000, 12.0, 2.4, 52, plant_size=25, plant_prob=0.85)[:3],
    "rmat2k": lambda: synth.rmat(2048, 16, 53, plant_size=20, plant_prob=1.0)[:3],
    # enough pairs for every block of the grid to take several tiles
    "chunglu12k": lambda: synth.chung_lu(12000, 14.0, 2.4, 54, plant_size=28, plant_prob=0.9)[:3],
}


def _oracle_r(n, s, d, k, T):
    off, adj = O.csr(n, s, d)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    return O.fw_sync(n, O.sct(n, off, adj, rank, vert, k), k, T)


def _run(sct, n, T, prec, flags, state=None):
    launches = K.kdss_kernel_launches()
    st = K.kdss_fw_iterate(sct, state, T, K.make_opts(precision=prec, flags=flags))
    r, t = K.kdss_state_copy_r(st, n, prec)
    return st, r.astype(np.uint64), t, K.kdss_kernel_launches() - launches


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [3, 5])
def test_resident_equals_the_oracle_and_the_per_iteration_launches(name, k):
    n, s, d = GRAPHS[name]()
    T = 17
    want = _oracle_r(n, s, d, k, T)
    sct = K.kdss_build_sct(n, s, d, k)
    info = K.kdss_sct_info(sct)
    assert info["pairs_per_class"][3:] == [0, 0]
    for prec in (K.KDSS_INT64, K.KDSS_FP64):
        _, res, t, nl = _run(sct, n, T, prec, 0)
        assert t == T
        _, per, _, nl2 = _run(sct, n, T, prec, K.KDSS_FLAG_PER_ITERATION)
        if info["eta_k"] > 0:   # (G1 holds no 5-clique: nothing to launch)
            assert nl <= 3, nl  # the planning kernel and one resident launch
            assert nl2 >= 2 * T
        assert np.array_equal(res, want), prec
        assert np.array_equal(per, want), prec


@pytest.mark.parametrize("prec", [K.KDSS_INT64, K.KDSS_FP64])
def test_resident_runs_continue_across_calls(prec):
    n, s, d = GRAPHS["chunglu3k"]()
    k = 4
    sct = K.kdss_build_sct(n, s, d, k)
    st = None
    for i, T in enumerate((1, 6, 2, 11)):   # odd and even lengths: r ends in either copy
        st, r, t, nl = _run(sct, n, T, prec, 0, st)
        assert nl <= 3 if i == 0 else nl == 1   # shares planned once per (state, SCT)
    assert t == 20
    assert np.array_equal(r, _oracle_r(n, s, d, k, 20))
    # a per-iteration call continues the same state
    st, r, t, _ = _run(sct, n, 5, prec, K.KDSS_FLAG_PER_ITERATION, st)
    assert t == 25 and np.array_equal(r, _oracle_r(n, s, d, k, 25))


def test_resident_at_k_on_a_k_agnostic_sct():
    n, s, d = GRAPHS["rmat2k"]()
    multi = K.kdss_build_sct_multi(n, s, d, 6)
    for k in (3, 5):
        st = K.kdss_fw_iterate_at(multi, k, None, 10, K.make_opts())
        r, _ = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
        assert np.array_equal(r, _oracle_r(n, s, d, k, 10))


@pytest.mark.parametrize("name", ["chunglu3k", "chunglu12k"])
def test_resident_extraction_and_timing(name):
    n, s, d = GRAPHS[name]()
    k, T = 5, 40
    sct = K.kdss_build_sct(n, s, d, k)
    o = K.make_opts(precision=K.KDSS_FP64, flags=K.KDSS_FLAG_PROFILE)
    st = K.kdss_fw_iterate(sct, None, T, o)
    tm = K.kdss_state_timing(st)
    assert tm["fw_launches"] == T and tm["fw_kernel_ms"] > 0
    res = K.kdss_extract(sct, st)
    st2 = K.kdss_fw_iterate(sct, None, T, K.make_opts(precision=K.KDSS_FP64,
                                                       flags=K.KDSS_FLAG_PER_ITERATION))
    res2 = K.kdss_extract(sct, st2)
    for key in ("istar", "count", "upper_bound", "rho_prime"):
        assert res[key] == res2[key], key
    assert res["ids"].tolist() == res2["ids"].tolist()
    if name == "chunglu3k":
        want = O.solve(n, s, d, k, T)
        assert (res["istar"], res["count"]) == (want["istar"], want["count"])
        assert res["ids"].tolist() == want["ids"].tolist()


def test_resident_solve_with_a_stop_rule():
    """kdss_solve with check_every runs the iterations in pieces between stop
    tests; the result equals the per-iteration form."""
    n, s, d = GRAPHS["chunglu3k"]()
    k, T = 4, 60
    a = K.kdss_solve(n, s, d, k, T, K.make_opts(precision=K.KDSS_FP64, check_every=7,
                                                 eps_stop=1e-3))
    b = K.kdss_solve(n, s, d, k, T, K.make_opts(precision=K.KDSS_FP64, check_every=7, eps_stop=1e-3,
                                                 flags=K.KDSS_FLAG_PER_ITERATION))
    assert (a["istar"], a["count"], a["t_used"]) == (b["istar"], b["count"], b["t_used"])
    assert a["upper_bound"] == b["upper_bound"]


@pytest.mark.parametrize("prec", [K.KDSS_INT64, K.KDSS_FP64])
def test_resident_levels_past_32_bits(prec):
    """A 30-clique beside a sparse graph at k = 10: c_k = C(30, 10) + ... so
    40 iterations keep every level below 2^31 (the launch runs on 32-bit
    levels) and the next 40 cross it (64-bit levels); both runs, and their
    hand-over inside one state, equal the oracle."""
    n1, s1, d1 = synth.chung_lu(1500, 8.0, 2.5, 61)[:3]
    iu = np.triu_indices(30, 1)
    n, s, d = n1 + 30, np.concatenate([s1, iu[0] + n1]).astype(np.int32), \
        np.concatenate([d1, iu[1] + n1]).astype(np.int32)
    k = 10
    sct = K.kdss_build_sct(n, s, d, k)
    info = K.kdss_sct_info(sct)
    ck = info["c_k"]
    assert 40 * ck < 2 ** 31 <= 80 * ck
    assert info["pairs_per_class"][3:] == [0, 0]
    st, r, t, nl = _run(sct, n, 40, prec, 0)
    assert nl <= 3 and np.array_equal(r, _oracle_r(n, s, d, k, 40))
    st, r, t, nl = _run(sct, n, 40, prec, 0, st)
    assert nl == 1 and t == 80
    assert np.array_equal(r, _oracle_r(n, s, d, k, 80))


def _oracle_cont_step(n, sct_o, k, prev, t):
    """One FP64 iteration of the continuous rule from r-hat_{t-1} = prev."""
    return O.fw_cont(n, sct_o, k, 1, r0=prev * (t - 1)) / t


@pytest.mark.parametrize("name", ["er300", "chunglu3k", "rmat2k", "chunglu12k"])
def test_resident_fp32_matches_the_fp64_oracle_per_iteration(name):
    """The continuous rule in the resident launch (FP32 r-hat with compensated
    shared-memory and global sums): one launch of one iteration from the
    GPU's own state equals one FP64 oracle iteration within 1e-5 (relative,
    inf-norm) at several horizons, across launches of several iterations; the
    per-iteration kernels reach the same density; sum r-hat = c_k."""
    n, s, d = GRAPHS[name]()
    k = 4
    off, adj = O.csr(n, s, d)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    so = O.sct(n, off, adj, rank, vert, k)
    sct = K.kdss_build_sct(n, s, d, k)
    ck = K.kdss_sct_info(sct)["c_k"]
    o = K.make_opts(precision=K.KDSS_FP32K, flags=K.KDSS_FLAG_PROFILE)
    st, done = None, 0
    for chunk in (1, 5, 1, 13, 1):
        prev = (K.kdss_state_copy_r(st, n, K.KDSS_FP32K)[0].astype(np.float64) if st
                else np.zeros(n))
        st = K.kdss_fw_iterate(sct, st, chunk, o)
        done += chunk
        got, t = K.kdss_state_copy_r(st, n, K.KDSS_FP32K)
        assert t == done
        if chunk == 1:
            want = _oracle_cont_step(n, so, k, prev, t)
            err = np.max(np.abs(got.astype(np.float64) - want)) / max(np.max(np.abs(want)), 1e-300)
            assert err <= 1e-5, (t, err)
        assert abs(float(got.astype(np.float64).sum()) - ck) <= 1e-5 * ck
    tm = K.kdss_state_timing(st)
    assert tm["fw_launches"] == done          # the resident launch counts every iteration
    per = K.kdss_fw_iterate(sct, None, done,
                            K.make_opts(precision=K.KDSS_FP32K, flags=K.KDSS_FLAG_PER_ITERATION))
    a, b = K.kdss_extract(sct, st), K.kdss_extract(sct, per)
    assert abs(a["density"] - b["density"]) <= 0.01 * b["density"]
