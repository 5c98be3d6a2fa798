"""The allocation-free FW entry point (kdss_fw_iterate_noalloc).

It serves callers that cannot allocate device memory while they iterate (a
pre-reserved memory arena, a fixed serving footprint, no synchronising
cudaMalloc between their kernels): the caller owns r and the library's fixed
scratch array holds the rest.  Its result must equal kdss_fw_iterate's
(integer rule, exact), call after call, although every call reuses the same
scratch array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)
    return torch


def _r_of(tensor):
    return tensor.cpu().numpy().view(np.uint64)


def _oracle_r(n, s, d, k, T):
    """r_T of the oracle's synchronous iterations (rule I) on its own SCT."""
    off, adj = O.csr(n, s, d)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    return O.fw_sync(n, O.sct(n, off, adj, rank, vert, k), k, T)


def test_noalloc_matches_fw_iterate_on_consecutive_calls(torch_cuda):
    torch = torch_cuda
    n, s, d, _ = synth.chung_lu(3000, 12.0, 2.4, 9, plant_size=25, plant_prob=0.85)
    k, T = 4, 25
    sct = K.kdss_build_sct(n, s, d, k)
    ref_T = K.kdss_state_copy_r(K.kdss_fw_iterate(sct, None, T), n, K.KDSS_INT64)[0]
    ref_2T = K.kdss_state_copy_r(K.kdss_fw_iterate(sct, None, 2 * T), n, K.KDSS_INT64)[0]
    # the existing entry point and the oracle agree, so both calls below are
    # checked against the oracle as well
    assert np.array_equal(ref_T, _oracle_r(n, s, d, k, T))
    assert np.array_equal(ref_2T, _oracle_r(n, s, d, k, 2 * T))
    r = torch.zeros(n, dtype=torch.int64, device="cuda")
    K.kdss_fw_iterate_noalloc(sct, r, 0, T)                  # first call
    assert np.array_equal(_r_of(r), ref_T)
    K.kdss_fw_iterate_noalloc(sct, r, T, T)                  # second call, right after
    assert np.array_equal(_r_of(r), ref_2T)
    r2 = torch.zeros(n, dtype=torch.int64, device="cuda")   # a fresh r: stale scratch cleared
    K.kdss_fw_iterate_noalloc(sct, r2, 0, T)
    assert np.array_equal(_r_of(r2), ref_T)


def test_noalloc_on_the_benchmark_graph(torch_cuda):
    torch = torch_cuda
    n, s, d = synth.workload_chunglu_1e5()
    k, T = 5, 20
    sct = K.kdss_build_sct(n, s, d, k)
    ref = K.kdss_state_copy_r(K.kdss_fw_iterate(sct, None, T), n, K.KDSS_INT64)[0]
    for _ in range(2):
        r = torch.zeros(n, dtype=torch.int64, device="cuda")
        K.kdss_fw_iterate_noalloc(sct, r, 0, T)
        assert np.array_equal(_r_of(r), ref)


def test_noalloc_rejects_inputs_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    n = 2_500_000                          # 8 n bytes of delta alone exceed 16 MiB
    src = np.array([0, 1, 2], np.int32)
    dst = np.array([1, 2, 0], np.int32)
    sct = K.kdss_build_sct(n, src, dst, 3)
    r = torch.zeros(n, dtype=torch.int64, device="cuda")
    with pytest.raises(K.KdssError) as e:
        K.kdss_fw_iterate_noalloc(sct, r, 0, 1)
    assert e.value.code == K.KDSS_ERR_INVALID_ARG
    assert "at most" in str(e.value) and "scratch" in str(e.value)
    # the entry point stays usable afterwards
    n2, s2, d2 = synth.g1()
    sct2 = K.kdss_build_sct(n2, s2, d2, 3)
    r2 = torch.zeros(n2, dtype=torch.int64, device="cuda")
    K.kdss_fw_iterate_noalloc(sct2, r2, 0, 10)
    ref = K.kdss_state_copy_r(K.kdss_fw_iterate(sct2, None, 10), n2, K.KDSS_INT64)[0]
    assert np.array_equal(_r_of(r2), ref)


def test_noalloc_rejects_r_outside_device_memory(torch_cuda):
    """A host buffer, a CPU tensor or a tensor shorter than n is refused with
    INVALID_ARG before any kernel runs, and the entry point stays usable."""
    torch = torch_cuda
    n, s, d = synth.g1()
    sct = K.kdss_build_sct(n, s, d, 3)
    host = np.zeros(n, np.uint64)
    with pytest.raises(K.KdssError) as e:        # raw host pointer: checked by the library
        K.kdss_fw_iterate_noalloc(sct, host.ctypes.data, 0, 1)
    assert e.value.code == K.KDSS_ERR_INVALID_ARG and "device memory" in str(e.value)
    with pytest.raises(K.KdssError) as e:        # CPU tensor
        K.kdss_fw_iterate_noalloc(sct, torch.zeros(n, dtype=torch.int64), 0, 1)
    assert e.value.code == K.KDSS_ERR_INVALID_ARG
    with pytest.raises(K.KdssError) as e:        # too short
        K.kdss_fw_iterate_noalloc(sct, torch.zeros(n - 1, dtype=torch.int64, device="cuda"), 0, 1)
    assert e.value.code == K.KDSS_ERR_INVALID_ARG
    assert not host.any()
    r = torch.zeros(n, dtype=torch.int64, device="cuda")
    K.kdss_fw_iterate_noalloc(sct, r, 0, 10)
    assert np.array_equal(_r_of(r), _oracle_r(n, s, d, 3, 10))
