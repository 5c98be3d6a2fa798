"""The k-agnostic SCT (kdss_build_sct_multi) and its restriction to one k.

By Lemma 2.5, P_k is P without the pairs with |V_h| > k or |V(P)| < k, and
the pivot choices of the recursion do not depend on k; so the restriction of
one k-agnostic build must give, for every k up to its k_max, exactly the
pairs that the k-pruned build emits (and the oracle's SCT), the same c_k,
and the same FW ranking.
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


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_restriction_equals_the_k_pruned_build(name):
    n, s, d = GRAPHS[name]()
    kmax = 7
    multi = K.kdss_build_sct_multi(n, s, d, kmax)
    info = K.kdss_sct_info(multi)
    assert info["k"] == kmax
    assert info["c_k"] == K.kdss_sct_info(K.kdss_build_sct(n, s, d, kmax))["c_k"]
    off, adj = O.csr(n, s, d)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    for k in range(2, kmax + 1):
        a = K.kdss_sct_restrict(multi, k)
        b = K.kdss_build_sct(n, s, d, k)
        assert gpu_pairs(a) == gpu_pairs(b) == O.canonical_pairs(O.sct(n, off, adj, rank, vert, k))
        ia, ib = K.kdss_sct_info(a), K.kdss_sct_info(b)
        assert (ia["c_k"], ia["eta_k"], ia["L_k"], ia["k"]) == (ib["c_k"], ib["eta_k"], ib["L_k"], k)
        if ia["eta_k"]:
            ra, _ = K.kdss_state_copy_r(K.kdss_fw_iterate(a, None, 20), n, K.KDSS_INT64)
            rb, _ = K.kdss_state_copy_r(K.kdss_fw_iterate(b, None, 20), n, K.KDSS_INT64)
            assert np.array_equal(ra, rb)


def test_k_agnostic_handles_are_restricted_before_use():
    n, s, d = synth.g1()
    multi = K.kdss_build_sct_multi(n, s, d, 4)
    for call in (lambda: K.kdss_fw_iterate(multi, None, 3),
                 lambda: K.kdss_sct_restrict(multi, 5),
                 lambda: K.kdss_sct_restrict(K.kdss_build_sct(n, s, d, 3), 3)):
        with pytest.raises(K.KdssError) as e:
            call()
        assert e.value.code == K.KDSS_ERR_INVALID_ARG


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_iterating_at_k_filters_p_k_in_place(name):
    """kdss_fw_iterate_at runs the iterations over P_k of the k-agnostic SCT
    where it stands (pairs outside P_k skipped by the kernels): r_T, c_k and
    the extracted prefix equal the k-pruned build's, bit for bit, in the
    integer rule, and the FP32 rule reaches the same density."""
    n, s, d = GRAPHS[name]()
    kmax, T = 7, 20
    multi = K.kdss_build_sct_multi(n, s, d, kmax)
    for k in range(2, kmax + 1):
        b = K.kdss_build_sct(n, s, d, k)
        if not K.kdss_sct_info(b)["eta_k"]:
            continue
        for prec in (K.KDSS_INT64, K.KDSS_FP64):
            o = K.make_opts(precision=prec)
            sa = K.kdss_fw_iterate_at(multi, k, None, T, o)
            sb = K.kdss_fw_iterate(b, None, T, o)
            ra, ta = K.kdss_state_copy_r(sa, n, prec)
            rb, tb = K.kdss_state_copy_r(sb, n, prec)
            assert ta == tb == T and np.array_equal(ra, rb), (k, prec)
            ea, eb = K.kdss_extract(multi, sa, o), K.kdss_extract(b, sb, o)
            assert (ea["istar"], ea["count"], ea["ids"].tolist()) == \
                (eb["istar"], eb["count"], eb["ids"].tolist())
            assert ea["upper_bound"] == eb["upper_bound"] and ea["rho_prime"] == eb["rho_prime"]
        o32 = K.make_opts(precision=K.KDSS_FP32K)
        ea = K.kdss_extract(multi, K.kdss_fw_iterate_at(multi, k, None, T, o32), o32)
        eb = K.kdss_extract(b, K.kdss_fw_iterate(b, None, T, o32), o32)
        assert abs(ea["density"] - eb["density"]) <= 0.01 * max(eb["density"], 1e-30)


def test_iterating_at_k_checks_its_arguments():
    n, s, d = synth.g1()
    multi = K.kdss_build_sct_multi(n, s, d, 4)
    pruned = K.kdss_build_sct(n, s, d, 3)
    st = K.kdss_fw_iterate_at(multi, 3, None, 2)
    for call in (lambda: K.kdss_fw_iterate_at(multi, 5, None, 1),       # above k_max
                 lambda: K.kdss_fw_iterate_at(multi, 1, None, 1),
                 lambda: K.kdss_fw_iterate_at(pruned, 4, None, 1),      # not its k
                 lambda: K.kdss_fw_iterate_at(multi, 4, st, 1)):        # a state of k = 3
        with pytest.raises(K.KdssError) as e:
            call()
        assert e.value.code == K.KDSS_ERR_INVALID_ARG
    st = K.kdss_fw_iterate_at(multi, 3, st, 48)
    res = K.kdss_extract(multi, st)
    assert res["istar"] == 6 and res["count"] == 8                      # Example 1.1
