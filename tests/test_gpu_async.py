"""In-place (asynchronous) FW iterations, KDSS_FLAG_ASYNC.

Pairs add their allocations straight into r while other pairs read it, as
Alg. 2 as printed updates r in place; the result depends on the schedule, so
the checks are the facts that hold for every schedule: each pair hands out
exactly n_C units within its caps (Lemma 2.6), so sum_u r_t(u) = t c_k
exactly and r_t(u) <= t cnt_k(u) (Lemma 3.1); r_t / t is feasible, so
rho'(V_i) of every prefix is below max r / t (Thms 3.5-3.6); the extracted
prefix's clique count is exact; and the density reaches the oracle's.
"""
import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)


GRAPHS = {
    "g1": lambda: (*synth.g1(), 3),
    "er300": lambda: (*synth.erdos_renyi(300, 0.06, 21), 3),
    "chunglu3k": lambda: (*synth.chung_lu(3000, 12.0, 2.4, 9, plant_size=25, plant_prob=0.85)[:3], 4),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("prec", [K.KDSS_INT64, K.KDSS_FP64])
def test_in_place_iterations_keep_the_invariants(name, prec):
    n, s, d, k = GRAPHS[name]()
    T = 60
    o = K.make_opts(precision=prec, flags=K.KDSS_FLAG_ASYNC)
    sct = K.kdss_build_sct(n, s, d, k)
    ck = K.kdss_sct_info(sct)["c_k"]
    st = K.kdss_fw_iterate(sct, None, T // 2, o)
    st = K.kdss_fw_iterate(sct, st, T - T // 2, o)       # resumed
    r, t = K.kdss_state_copy_r(st, n, prec)
    r = r.astype(np.uint64)
    assert t == T and int(r.sum()) == T * ck                      # Lemma 3.1, exact
    off, adj = O.csr(n, s, d)
    cl = O.list_cliques(n, off, adj, k)
    cnt = np.bincount(cl.ravel(), minlength=n) if len(cl) else np.zeros(n, np.int64)
    assert np.all(r <= T * cnt.astype(np.uint64))                 # r_t(u) <= t cnt_k(u)
    res = K.kdss_extract(sct, st)
    assert res["rho_prime"] <= res["upper_bound"] * (1 + 1e-12)   # weak duality
    if res["istar"]:
        inside = np.zeros(n, bool)
        inside[res["ids"]] = True
        keep = inside[s] & inside[d]
        o2, a2 = O.csr(n, s[keep], d[keep])
        assert res["count"] == O.count_cliques(n, o2, a2, k)
    want = O.solve(n, s, d, k, T)["density"]
    assert res["density"] >= 0.99 * want


def test_in_place_iterations_need_the_integer_rule():
    n, s, d = synth.g1()
    sct = K.kdss_build_sct(n, s, d, 3)
    with pytest.raises(K.KdssError) as e:
        K.kdss_fw_iterate(sct, None, 5, K.make_opts(precision=K.KDSS_FP32K, flags=K.KDSS_FLAG_ASYNC))
    assert e.value.code == K.KDSS_ERR_UNSUPPORTED
