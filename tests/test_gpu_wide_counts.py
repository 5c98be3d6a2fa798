"""Clique counts beyond 64 bits on the GPU (Lemma 2.6 counts kept exact in
128 bits).

Pairs of 60 to 130 nodes with k = 40 have n_C = C(p, k - h) far above 2^64.
Through kdss_sct_from_pairs the SCT's c_k must equal the exact sum (Python
integers), the integer rule must refuse the iterations (r would leave its
exact range), the FP32 continuous rule must match the FP64 oracle (whose
counts come from its own 128-bit binomials), and the extracted prefix count
must equal the exact count of the oracle for the same node order.
"""
import math
import random

import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)


def _wide_pairs(seed, k=40, n=600, npairs=40):
    rng = random.Random(seed)
    po, nodes, h = [0], [], []
    for q in range(npairs):
        hh = rng.randint(1, 4)
        ln = rng.randint(max(k, 60), 130) if q % 3 else rng.randint(k, 50)
        sel = rng.sample(range(n), ln)
        nodes += sel
        h.append(hh)
        po.append(len(nodes))
    return n, {"pair_off": np.array(po, np.int64), "nodes": np.array(nodes, np.int32),
               "h": np.array(h, np.int32)}


def _exact_ck(sc, k):
    po, h = sc["pair_off"], sc["h"]
    return sum(math.comb(int(po[q + 1] - po[q] - h[q]), k - int(h[q])) for q in range(len(h)))


@pytest.mark.parametrize("seed", [1, 2])
def test_counts_beyond_64_bits(seed):
    k = 40
    n, sc = _wide_pairs(seed, k)
    want_ck = _exact_ck(sc, k)
    assert want_ck >= 2 ** 64
    s = K.kdss_sct_from_pairs(n, k, sc["pair_off"], sc["nodes"], sc["h"])
    info = K.kdss_sct_info(s)
    assert info["c_k"] == want_ck

    # the integer rule cannot hold r exactly
    for prec in (K.KDSS_INT64, K.KDSS_FP64):
        with pytest.raises(K.KdssError) as e:
            K.kdss_fw_iterate(s, None, 1, K.make_opts(precision=prec))
        assert e.value.code == K.KDSS_ERR_OVERFLOW

    # FP32 continuous rule against the FP64 oracle
    o32 = K.make_opts(precision=K.KDSS_FP32K)
    for T in (1, 3):
        st = K.kdss_fw_iterate(s, None, T, o32)
        r32, t = K.kdss_state_copy_r(st, n, K.KDSS_FP32K)
        assert t == T
        r64 = O.fw_cont(n, sc, k, T) / T
        err = np.max(np.abs(r32.astype(np.float64) - r64)) / np.max(np.abs(r64))
        assert err <= FP32_RTOL, err
        assert abs(float(r32.astype(np.float64).sum()) - want_ck) <= FP32_RTOL * want_ck

    # extraction with 128-bit prefix counts: the GPU's order is (r desc, id
    # asc) on its own float r; the oracle counts every prefix of that order
    res = K.kdss_extract(s, st, o32)
    order = np.lexsort((np.arange(n), -r32.astype(np.float64))).astype(np.int32)
    lo, hi, flo, fhi = O.prefix_counts_pairs(n, order, sc, k)
    i = O.argmax_density(lo, hi)
    assert res["istar"] == i
    assert res["count"] == int(lo[i]) | (int(hi[i]) << 64)
    assert res["count"] >= 2 ** 64
    assert res["ids"].tolist() == sorted(order[:i].tolist())
