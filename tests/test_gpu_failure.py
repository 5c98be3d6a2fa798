"""Failure detection on the GPU without a fault: a bounded device wait that
runs out is reported as KDSS_ERR_TIMEOUT and leaves the context usable.

KDSS_FLAG_TEST_BARRIER_TIMEOUT makes the peeling kernel's grid barriers wait
for one block more than the grid holds, with a 1 ms limit: no block can pass
its first barrier, every block gives up after its own limit and returns, and
the host reads the timeout from the device error word.  No trap, no bad
address and no endless loop is involved.
"""
import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)
    return K


def test_expired_barrier_wait_is_reported_and_the_library_stays_usable(lib):
    n, s, d, _ = synth.chung_lu(3000, 10.0, 2.4, 31, plant_size=20, plant_prob=0.9)
    k, T = 4, 12
    bad = K.make_opts(flags=K.KDSS_FLAG_TEST_BARRIER_TIMEOUT)
    for _ in range(2):
        with pytest.raises(K.KdssError) as e:
            K.kdss_build_sct(n, s, d, k, bad)
        assert e.value.code == K.KDSS_ERR_TIMEOUT
        assert "barrier" in str(e.value)
    with pytest.raises(K.KdssError) as e:
        K.kdss_solve(n, s, d, k, T, bad)
    assert e.value.code == K.KDSS_ERR_TIMEOUT
    # the same process and context go on to solve correctly
    sct = K.kdss_build_sct(n, s, d, k)
    st = K.kdss_fw_iterate(sct, None, T)
    r, _ = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
    want = O.solve(n, s, d, k, T)
    assert np.array_equal(r, want["r"])
    res = K.kdss_extract(sct, st)
    assert res["istar"] == want["istar"] and res["count"] == want["count"]
