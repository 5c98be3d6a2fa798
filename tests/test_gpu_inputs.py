"""Where the caller's arrays live.

Arrays passed as device memory (a graph descriptor with on_device = 1, the
device pair arrays of kdss_sct_from_pairs, device edge lists of batch and
server queries) are checked with cudaPointerGetAttributes before any kernel
runs: a host pointer is refused with KDSS_ERR_INVALID_ARG instead of reaching
a kernel.  The binding checks both edge tensors (dtype, layout, length,
device) and sends CPU tensors down the host path.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K
import synth


def test_cpu_tensors_take_the_host_path():
    torch = pytest.importorskip("torch")
    n, s, d = synth.g1()
    g, keep = K._graph_desc(n, torch.from_numpy(np.asarray(s, np.int32)), np.asarray(d, np.int32))
    assert g.on_device == 0 and g.m == len(s) and g.n == n
    assert np.array_equal(np.ctypeslib.as_array(C.cast(g.src, C.POINTER(C.c_int32)), (g.m,)), s)
    with pytest.raises(ValueError):
        K._graph_desc(n, np.asarray(s[:-1], np.int32), np.asarray(d, np.int32))


def test_pair_arrays_of_unequal_lengths_are_refused_on_the_host():
    po, nodes, h = np.array([0, 3], np.int64), np.array([0, 1, 2], np.int32), np.array([1], np.int32)
    for args in ((po[:1], nodes, h), (po, nodes[:2], h), (po + 1, nodes, h), (po, nodes, h[:0])):
        with pytest.raises(ValueError):
            K.kdss_sct_from_pairs(3, 2, *args)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)
    return torch


def _g1_arrays():
    n, s, d = synth.g1()
    return n, np.ascontiguousarray(s, np.int32), np.ascontiguousarray(d, np.int32)


def _g1_ids():
    """{u1..u6} of Example 1.1, as the oracle numbers them."""
    n, s, d = _g1_arrays()
    return sorted(O.solve(n, s, d, 3, 100)["ids"].tolist())


def _g1_still_solves():
    n, s, d = _g1_arrays()
    res = K.kdss_solve(n, s, d, 3, 100)
    assert sorted(res["ids"].tolist()) == _g1_ids()
    assert abs(res["density"] - 4.0 / 3.0) < 1e-12


@pytest.mark.gpu
def test_host_pointers_passed_as_device_edges_are_refused(torch_cuda):
    torch = torch_cuda
    L = K.load()
    n, s, d = _g1_arrays()
    dev_s = torch.from_numpy(s).cuda()
    for src, dst in ((s.ctypes.data, d.ctypes.data), (dev_s.data_ptr(), d.ctypes.data)):
        g = K.kdss_graph_desc(n=n, m=s.size, src=src, dst=dst, on_device=1)
        out = C.c_void_p()
        rc = L.kdss_build_sct(C.byref(g), 3, C.byref(K.make_opts()), C.byref(out))
        assert rc == K.KDSS_ERR_INVALID_ARG and not out.value
        assert b"device memory" in L.kdss_last_error()
        r = K.kdss_result()
        rc = L.kdss_solve(C.byref(g), 3, 10, C.byref(K.make_opts()), C.byref(r))
        assert rc == K.KDSS_ERR_INVALID_ARG
        L.kdss_result_free(C.byref(r))
        # a batch refuses that query alone
        q = (K.kdss_query * 2)()
        q[0].graph, q[0].k, q[0].T = g, 3, 10
        ok = K.kdss_graph_desc(n=n, m=s.size, src=s.ctypes.data, dst=d.ctypes.data, on_device=0)
        q[1].graph, q[1].k, q[1].T = ok, 3, 100
        res = (K.kdss_result * 2)()
        rc = L.kdss_solve_batch(q, 2, res, C.byref(K.make_opts()))
        assert rc == K.KDSS_ERR_INVALID_ARG
        assert res[0].status == K.KDSS_ERR_INVALID_ARG and res[1].status == K.KDSS_OK
        assert abs(res[1].density - 4.0 / 3.0) < 1e-12
        for i in range(2):
            L.kdss_result_free(C.byref(res[i]))
    _g1_still_solves()


@pytest.mark.gpu
def test_host_pair_arrays_passed_as_device_memory_are_refused(torch_cuda):
    L = K.load()
    pair_off = np.array([0, 3], np.int64)
    nodes = np.array([0, 1, 2], np.int32)
    h = np.array([3], np.int32)
    out = C.c_void_p()
    rc = L.kdss_sct_from_pairs(3, 3, 1, pair_off.ctypes.data, nodes.ctypes.data, h.ctypes.data, 1,
                               C.byref(K.make_opts()), C.byref(out))
    assert rc == K.KDSS_ERR_INVALID_ARG and not out.value
    assert b"pair_off" in L.kdss_last_error()
    _g1_still_solves()


@pytest.mark.gpu
def test_server_refuses_host_pointers_passed_as_device_edges(torch_cuda):
    L = K.load()
    n, s, d = _g1_arrays()
    with K.Server() as srv:
        q = K.kdss_query()
        q.graph = K.kdss_graph_desc(n=n, m=s.size, src=s.ctypes.data, dst=d.ctypes.data, on_device=1)
        q.k, q.T = 3, 10
        t = C.c_int64()
        rc = L.kdss_server_submit(srv.ptr, C.byref(q), C.byref(t))
        assert rc == K.KDSS_ERR_INVALID_ARG
        res = srv.wait(srv.submit(n, s, d, 3, 100))
        assert abs(res["density"] - 4.0 / 3.0) < 1e-12


@pytest.mark.gpu
def test_binding_checks_both_edge_tensors(torch_cuda):
    torch = torch_cuda
    n, s, d = _g1_arrays()
    ds, dd = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    with pytest.raises(ValueError):                 # dst on the host, src on the device
        K.kdss_build_sct(n, ds, torch.from_numpy(d), 3)
    with pytest.raises(ValueError):                 # dst shorter than src
        K.kdss_build_sct(n, ds, dd[:-1].contiguous(), 3)
    with pytest.raises(ValueError):                 # wrong dtype
        K.kdss_build_sct(n, ds, dd.to(torch.int64), 3)
    want = _g1_ids()
    res = K.kdss_solve(n, ds, dd, 3, 100)           # both on the device
    assert sorted(res["ids"].tolist()) == want
    res = K.kdss_solve(n, torch.from_numpy(s), torch.from_numpy(d), 3, 100)   # CPU tensors
    assert sorted(res["ids"].tolist()) == want


@pytest.mark.gpu
def test_rule_option_is_checked_against_the_precision(torch_cuda):
    """kdss_opts.rule: the default and the matching rule give the precision's
    rule; a rule the precision does not hold, or an unknown one, is refused."""
    n, s, d = _g1_arrays()
    sct = K.kdss_build_sct(n, s, d, 3)
    base = K.kdss_state_copy_r(K.kdss_fw_iterate(sct, None, 20), n, K.KDSS_INT64)[0]
    st = K.kdss_fw_iterate(sct, None, 20, K.make_opts(rule=K.KDSS_RULE_INTEGER))
    assert np.array_equal(K.kdss_state_copy_r(st, n, K.KDSS_INT64)[0], base)
    st = K.kdss_fw_iterate(sct, None, 100, K.make_opts(precision=K.KDSS_FP32K,
                                                       rule=K.KDSS_RULE_CONTINUOUS))
    assert abs(K.kdss_extract(sct, st)["density"] - 4.0 / 3.0) < 1e-12
    for prec, rule, code in ((K.KDSS_FP32K, K.KDSS_RULE_INTEGER, K.KDSS_ERR_UNSUPPORTED),
                             (K.KDSS_INT64, K.KDSS_RULE_CONTINUOUS, K.KDSS_ERR_UNSUPPORTED),
                             (K.KDSS_FP64, K.KDSS_RULE_CONTINUOUS, K.KDSS_ERR_UNSUPPORTED),
                             (K.KDSS_INT64, 7, K.KDSS_ERR_INVALID_ARG)):
        with pytest.raises(K.KdssError) as e:
            K.kdss_fw_iterate(sct, None, 5, K.make_opts(precision=prec, rule=rule))
        assert e.value.code == code
        with pytest.raises(K.KdssError) as e:
            K.kdss_solve(n, s, d, 3, 5, K.make_opts(precision=prec, rule=rule))
        assert e.value.code == code
    _g1_still_solves()

