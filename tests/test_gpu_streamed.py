"""The streamed solve (kdss_solve_streamed): the SCT rebuilt root range by
root range inside every iteration, for SCTs that do not fit the device.

In the synchronous reading every pair of iteration t reads r_{t-1} and the
integer allocations are summed, so splitting the pairs into root ranges
changes nothing: the result must equal the unsplit solve and the oracle bit
for bit (integer rule), for any number of ranges.
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
    "rmat2k": lambda: synth.rmat(2048, 16, 21, plant_size=20, plant_prob=1.0)[:3],
    "chunglu3k": lambda: synth.chung_lu(3000, 12.0, 2.4, 22, plant_size=25, plant_prob=0.85)[:3],
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [3, 5])
def test_streamed_equals_unsplit_and_oracle(name, k):
    n, s, d = GRAPHS[name]()
    T = 25
    want = O.solve(n, s, d, k, T)
    whole = K.kdss_solve(n, s, d, k, T)
    assert whole["istar"] == want["istar"] and whole["count"] == want["count"]
    for nchunks in (1, 3, 7, 64):
        for prec in (K.KDSS_INT64, K.KDSS_FP64):
            got = K.kdss_solve_streamed(n, s, d, k, T, nchunks, K.make_opts(precision=prec))
            assert got["istar"] == want["istar"], (nchunks, prec)
            assert got["ids"].tolist() == want["ids"].tolist()
            assert got["count"] == want["count"]
            assert got["upper_bound"] == whole["upper_bound"]
            assert got["rho_prime"] == whole["rho_prime"]
            assert got["t_used"] == T


def test_streamed_fp32_density_matches_oracle():
    n, s, d = GRAPHS["chunglu3k"]()
    k, T = 4, 40
    want = O.solve(n, s, d, k, T)
    got = K.kdss_solve_streamed(n, s, d, k, T, 5, K.make_opts(precision=K.KDSS_FP32K))
    assert abs(got["density"] - want["density"]) <= 0.01 * want["density"]
    assert got["gap"] >= -1e-6


def test_streamed_refuses_in_place_iterations_and_bad_chunks():
    n, s, d = synth.g1()
    with pytest.raises(K.KdssError) as e:
        K.kdss_solve_streamed(n, s, d, 3, 5, 2, K.make_opts(flags=K.KDSS_FLAG_ASYNC))
    assert e.value.code == K.KDSS_ERR_UNSUPPORTED
    with pytest.raises(K.KdssError) as e:
        K.kdss_solve_streamed(n, s, d, 3, 5, 0)
    assert e.value.code == K.KDSS_ERR_INVALID_ARG
    res = K.kdss_solve_streamed(n, s, d, 3, 50, 3)
    assert res["istar"] == 6 and res["count"] == 8
