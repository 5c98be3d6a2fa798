"""The prefix-shared form of an SCT (kdss_sct_share_prefixes).

Front coding changes how the pairs are stored, not which pairs there are:
the decoded pairs must be the flat SCT's pairs (and the oracle's), and in
the synchronous integer rule the FW iterations are a sum over pairs, so r_T,
the extracted prefix and its exact count must equal the flat handle's and
the oracle's bit for bit, for every chunk size the iterations decode.
"""
import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K
import synth
from test_gpu_parity import gpu_pairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)


GRAPHS = {
    "g1": synth.g1,
    "er300": lambda: synth.erdos_renyi(300, 0.06, 21),
    "chunglu3k": lambda: synth.chung_lu(3000, 12.0, 2.4, 9, plant_size=25, plant_prob=0.85)[:3],
    "rmat1500": lambda: synth.batch_rmat_graph(3, 1500),
}


def _oracle_sct(n, s, d, k):
    off, adj = O.csr(n, s, d)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    return O.sct(n, off, adj, rank, vert, k)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [3, 5])
def test_shared_pairs_are_the_flat_pairs(name, k):
    n, s, d = GRAPHS[name]()
    flat = K.kdss_build_sct(n, s, d, k)
    sh = K.kdss_sct_share_prefixes(flat, 64)
    fi, si = K.kdss_sct_info(flat), K.kdss_sct_info(sh)
    for key in ("eta_k", "L_k", "c_k", "k", "n", "max_pair_len"):
        assert fi[key] == si[key], key
    assert fi["pairs_per_class"] == si["pairs_per_class"]
    assert gpu_pairs(sh) == gpu_pairs(flat) == O.canonical_pairs(_oracle_sct(n, s, d, k))
    w = K.kdss_sct_shared_words(sh)
    assert 0 <= w["words"] <= fi["L_k"]
    if fi["eta_k"] > 64:
        assert w["chunks"] > 1 and w["words"] < fi["L_k"]


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("chunk", [32, 200, 0])
def test_shared_iterations_equal_flat_and_oracle(name, chunk):
    n, s, d = GRAPHS[name]()
    k, T = 4, 25
    flat = K.kdss_build_sct(n, s, d, k)
    if not K.kdss_sct_info(flat)["eta_k"]:
        pytest.skip("no 4-cliques")
    sh = K.kdss_sct_share_prefixes(flat, chunk)
    want = O.fw_sync(n, _oracle_sct(n, s, d, k), k, T)
    for prec in (K.KDSS_INT64, K.KDSS_FP64):
        o = K.make_opts(precision=prec)
        st = K.kdss_fw_iterate(sh, None, 10, o)
        st = K.kdss_fw_iterate(sh, st, T - 10, o)   # continued state
        r, t = K.kdss_state_copy_r(st, n, prec)
        rf, _ = K.kdss_state_copy_r(K.kdss_fw_iterate(flat, None, T, o), n, prec)
        if prec == K.KDSS_FP64:
            r = r.astype(np.uint64)
            rf = rf.astype(np.uint64)
        assert t == T
        assert np.array_equal(r, rf)
        assert np.array_equal(r, want)
        a, b = K.kdss_extract(sh, st), K.kdss_extract(flat, K.kdss_fw_iterate(flat, None, T, o))
        assert (a["istar"], a["count"]) == (b["istar"], b["count"])
        assert a["ids"].tolist() == b["ids"].tolist()
        assert a["upper_bound"] == b["upper_bound"]


def test_shared_k_agnostic_iterates_p_k_where_it_stands():
    n, s, d = GRAPHS["chunglu3k"]()
    kmax, T = 6, 15
    multi = K.kdss_build_sct_multi(n, s, d, kmax)
    sh = K.kdss_sct_share_prefixes(multi, 100)
    assert K.kdss_sct_shared_words(sh)["words"] < K.kdss_sct_info(multi)["L_k"]
    for k in range(3, kmax + 1):
        b = K.kdss_build_sct(n, s, d, k)
        if not K.kdss_sct_info(b)["eta_k"]:
            continue
        st = K.kdss_fw_iterate_at(sh, k, None, T)
        rs, _ = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
        rb, _ = K.kdss_state_copy_r(K.kdss_fw_iterate(b, None, T), n, K.KDSS_INT64)
        assert np.array_equal(rs, rb)
        es, eb = K.kdss_extract(sh, st), K.kdss_extract(b, K.kdss_fw_iterate(b, None, T))
        assert (es["istar"], es["count"]) == (eb["istar"], eb["count"])


def test_shared_fp32_rule_keeps_the_invariants():
    n, s, d = GRAPHS["chunglu3k"]()
    k, T = 4, 30
    flat = K.kdss_build_sct(n, s, d, k)
    sh = K.kdss_sct_share_prefixes(flat, 96)
    o = K.make_opts(precision=K.KDSS_FP32K)
    st = K.kdss_fw_iterate(sh, None, T, o)
    r, _ = K.kdss_state_copy_r(st, n, K.KDSS_FP32K)
    ck = K.kdss_sct_info(flat)["c_k"]
    assert abs(float(np.sum(r.astype(np.float64))) - ck) <= 1e-4 * ck   # r-hat sums to c_k
    a = K.kdss_extract(sh, st)
    b = K.kdss_extract(flat, K.kdss_fw_iterate(flat, None, T, o))
    assert abs(a["density"] - b["density"]) <= 0.01 * b["density"]


def test_shared_handles_refuse_calls_that_need_flat_pairs():
    n, s, d = synth.g1()
    flat = K.kdss_build_sct(n, s, d, 3)
    sh = K.kdss_sct_share_prefixes(flat)
    for call, code in ((lambda: K.kdss_sct_share_prefixes(sh), K.KDSS_ERR_INVALID_ARG),
                       (lambda: K.kdss_fw_cliques(sh, None, 3), K.KDSS_ERR_INVALID_ARG),
                       (lambda: K.kdss_fw_iterate(sh, None, 3, K.make_opts(flags=K.KDSS_FLAG_ASYNC)),
                        K.KDSS_ERR_UNSUPPORTED),
                       (lambda: K.kdss_sct_shared_words(flat), K.KDSS_ERR_INVALID_ARG)):
        with pytest.raises(K.KdssError) as e:
            call()
        assert e.value.code == code


def test_shared_on_the_benchmark_graph():
    """Chung-Lu n = 1e5, k = 5: the shared form keeps about half of the node
    words; its iterations equal the flat handle's and the oracle's."""
    n, s, d = synth.workload_chunglu_1e5()
    k, T = 5, 12
    flat = K.kdss_build_sct(n, s, d, k)
    sh = K.kdss_sct_share_prefixes(flat, 1 << 16)
    info = K.kdss_sct_info(flat)
    w = K.kdss_sct_shared_words(sh)
    assert w["chunks"] >= 2 and w["words"] < 0.6 * info["L_k"]
    o = K.make_opts(precision=K.KDSS_FP64)
    r, _ = K.kdss_state_copy_r(K.kdss_fw_iterate(sh, None, T, o), n, K.KDSS_FP64)
    rf, _ = K.kdss_state_copy_r(K.kdss_fw_iterate(flat, None, T, o), n, K.KDSS_FP64)
    assert np.array_equal(r, rf)
    assert np.array_equal(r.astype(np.uint64), O.fw_sync(n, _oracle_sct(n, s, d, k), k, T))
