"""Alg. 1 over the explicit k-clique list on the GPU (kdss_fw_cliques).

The list is expanded from the SCT on the device; it must be exactly the
oracle's explicit clique list (Lemmas 2.4-2.5: the pairs partition C_k(V)).
The synchronous Alg. 1 iterations must give the oracle's r_T bit for bit, and
the extraction on that state the oracle's prefix.
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
    "g1_k3": lambda: (*synth.g1(), 3),
    "er300_k3": lambda: (*synth.erdos_renyi(300, 0.06, 21), 3),
    "er120_k4": lambda: (*synth.erdos_renyi(120, 0.25, 22), 4),
    "chunglu3k_k4": lambda: (*synth.chung_lu(3000, 12.0, 2.4, 9, plant_size=25, plant_prob=0.85)[:3], 4),
    "rmat1500_k5": lambda: (*synth.batch_rmat_graph(3, 1500), 5),
    "clique7_k7": lambda: (7, *np.array([(a, b) for a in range(7) for b in range(a + 1, 7)],
                                         np.int32).T.copy(), 7),
}


def _rows(cl):
    return sorted(tuple(sorted(int(x) for x in row)) for row in cl)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_expansion_is_the_explicit_clique_list(name):
    n, s, d, k = GRAPHS[name]()
    sct = K.kdss_build_sct(n, s, d, k)
    got = K.kdss_sct_copy_cliques(sct)
    off, adj = O.csr(n, s, d)
    want = O.list_cliques(n, off, adj, k)
    assert got.shape == (len(want), k)
    assert _rows(got) == _rows(want)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_alg1_iterations_and_extraction_match_the_oracle(name):
    n, s, d, k = GRAPHS[name]()
    T = 40
    sct = K.kdss_build_sct(n, s, d, k)
    st = K.kdss_fw_cliques(sct, None, T // 4)
    st = K.kdss_fw_cliques(sct, st, T - T // 4)              # resumed
    r, t = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
    off, adj = O.csr(n, s, d)
    cl = O.list_cliques(n, off, adj, k)
    want = O.fw_cliques_sync(n, cl, k, T)
    assert t == T and np.array_equal(r, want)
    res = K.kdss_extract(sct, st)
    order = O.sort_desc(want)
    lo, hi = O.prefix_counts_cliques(n, order, cl, k)
    i = O.argmax_density(lo, hi)
    assert res["istar"] == i and res["count"] == int(lo[i])
    assert res["ids"].tolist() == sorted(order[:i].tolist())
    assert res["upper_bound"] == pytest.approx(float(want.max()) / T, rel=1e-12)


def test_alg1_needs_the_integer_state():
    n, s, d = synth.g1()
    sct = K.kdss_build_sct(n, s, d, 3)
    with pytest.raises(K.KdssError) as e:
        K.kdss_fw_cliques(sct, None, 3, K.make_opts(precision=K.KDSS_FP64))
    assert e.value.code == K.KDSS_ERR_UNSUPPORTED
