"""The continuous-batching server (include/kdss_server.h).

Queries of different graphs, k and T arrive while others are iterating; each
result must be the one kdss_solve returns for the query alone with the same
stop rule -- bit for bit for the integer rule, within the FP32 tolerance for
the continuous rule -- whatever the mix, the arrival order or the HBM budget
that decides how many queries are resident together.
"""
import threading
import time

import numpy as np
import pytest

import paper_2403_05775_gb300 as K
import synth

pytestmark = pytest.mark.gpu

FIELDS = ("istar", "count", "density", "upper_bound", "rho_prime", "gap", "T", "t_used")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)


def _queries():
    qs = []
    n, s, d = synth.g1()
    qs.append((n, s, d, 3, 40))
    for i, (nn, p, k) in enumerate([(300, 0.05, 3), (120, 0.2, 4), (800, 0.02, 3)]):
        n, s, d = synth.erdos_renyi(nn, p, 40 + i)
        qs.append((n, s, d, k, 60))
    for i, (nn, k, T) in enumerate([(3000, 4, 80), (5000, 5, 120), (2000, 6, 33), (8000, 3, 200)]):
        n, s, d, _ = synth.chung_lu(nn, 10.0, 2.5, 50 + i, plant_size=20, plant_prob=0.9)
        qs.append((n, s, d, k, T))
    n, s, d = synth.batch_rmat_graph(3, 1500)
    qs.append((n, s, d, 5, 50))
    qs.append((0, np.zeros(0, np.int32), np.zeros(0, np.int32), 3, 10))
    qs.append((7, *synth.g1()[1:], 3, 0))
    return qs


def _solo(q, prec, every, eps):
    return K.kdss_solve(*q, K.make_opts(precision=prec, check_every=every, eps_stop=eps))


def _same(a, b):
    for f in FIELDS:
        assert a[f] == b[f], (f, a[f], b[f])
    assert a["ids"].tolist() == b["ids"].tolist()


@pytest.mark.parametrize("prec", [K.KDSS_INT64, K.KDSS_FP64])
@pytest.mark.parametrize("budget", [0, 1])
def test_results_equal_each_query_alone(prec, budget):
    """budget 1 byte: one query resident at a time; 0: all of them."""
    qs = _queries()
    every, eps = 5, 0.02
    with K.Server(precision=prec, check_every=every, eps_stop=eps, hbm_budget=budget) as srv:
        tickets = [srv.submit(*q) for q in qs]
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(qs) and st["failed"] == 0
    if budget == 1:
        assert st["peak_active"] == 1
    else:
        assert st["peak_active"] > 1
    for q, g in zip(qs, got):
        assert g["status"] == K.KDSS_OK
        _same(g, _solo(q, prec, every, eps))
        assert g["timing"]["latency_ms"] >= g["timing"]["iterate_ms"] >= 0


def test_arrivals_during_iterations():
    """Queries submitted from another thread at random gaps while earlier
    ones iterate: same results as alone, later queries join running batches."""
    qs = _queries()
    every, eps = 5, 0.0
    rng = np.random.default_rng(7)
    tickets = [None] * len(qs)
    with K.Server(precision=K.KDSS_INT64, check_every=every, eps_stop=eps) as srv:
        def feed():
            for i in rng.permutation(len(qs)):
                tickets[i] = srv.submit(*qs[i])
                time.sleep(float(rng.exponential(0.004)))
        th = threading.Thread(target=feed)
        th.start()
        th.join()
        got = [srv.wait(t) for t in tickets]
    for q, g in zip(qs, got):
        _same(g, _solo(q, K.KDSS_INT64, every, eps))


def test_fp32_results_match_alone_within_tolerance():
    qs = _queries()[:9]
    every, eps = 5, 0.0
    with K.Server(precision=K.KDSS_FP32K, check_every=every) as srv:
        got = [srv.wait(t) for t in [srv.submit(*q) for q in qs]]
    for q, g in zip(qs, got):
        a = _solo(q, K.KDSS_FP32K, every, eps)
        assert g["t_used"] == a["t_used"] == q[4]
        if a["density"] > 0:
            # two FP32 runs sum their allocations in different orders (the
            # server's per-iteration kernels, the solo run's resident launch)
            # and the continuous rule's trajectory amplifies round-off (a
            # 1e-13 perturbation reaches ~2% by t = 80; at t = 33, k = 6 each
            # run's max r-hat is 1-9% from the FP64 oracle's), so the runs
            # agree on the extracted density, not on r or its maximum; each
            # run's bound holds for itself (weak duality)
            assert abs(g["density"] - a["density"]) <= 1e-2 * a["density"]
            assert g["rho_prime"] <= g["upper_bound"] * (1 + 1e-5)
            assert a["rho_prime"] <= a["upper_bound"] * (1 + 1e-5)


def test_errors_timeouts_and_tickets():
    n, s, d = synth.g1()
    with K.Server(check_every=3) as srv:
        with pytest.raises(K.KdssError) as e:
            srv.submit(n, s, d, 1, 10)
        assert e.value.code == K.KDSS_ERR_INVALID_ARG
        bad = srv.submit(5, np.array([0, 9], np.int32), np.array([1, 2], np.int32), 3, 10)
        big = srv.submit(*_queries()[7])
        ok = srv.submit(n, s, d, 3, 10)
        r = srv.wait(bad)
        assert r["status"] == K.KDSS_ERR_BAD_GRAPH and r["istar"] == 0
        r = srv.wait(ok)
        assert r["status"] == K.KDSS_OK and r["istar"] == 6 and r["t_used"] == 10
        try:
            srv.wait(big, timeout_ms=0)
        except K.KdssError as err:
            assert err.code == K.KDSS_ERR_TIMEOUT
        assert srv.wait(big)["status"] == K.KDSS_OK
        with pytest.raises(K.KdssError) as e:
            srv.wait(ok)                      # retired ticket
        assert e.value.code == K.KDSS_ERR_INVALID_ARG


def test_solve_stop_rule_matches_fixed_T_prefix():
    """kdss_solve with the stop rule runs a multiple of check_every (or T)
    iterations, and its result is that of a plain solve with that T."""
    n, s, d, _ = synth.chung_lu(5000, 10.0, 2.5, 51, plant_size=20, plant_prob=0.9)
    a = _solo((n, s, d, 5, 300), K.KDSS_INT64, 5, 0.02)
    assert a["t_used"] % 5 == 0 and a["t_used"] <= 300
    assert a["gap"] <= 0.02 or a["t_used"] == 300
    b = K.kdss_solve(n, s, d, 5, a["t_used"])
    for f in ("istar", "count", "upper_bound", "rho_prime", "gap"):
        assert a[f] == b[f]


def test_in_place_server_keeps_the_invariants():
    """KDSS_FLAG_ASYNC: queries iterate in place; the schedule decides the
    exact r, so the checks are the facts that hold for any schedule: every
    query runs T iterations (no stop rule), its bound covers its rho', and
    it extracts the density of the synchronous solve within 1%."""
    qs = _queries()[:9]
    with K.Server(precision=K.KDSS_INT64, check_every=5, flags=K.KDSS_FLAG_ASYNC) as srv:
        got = [srv.wait(t) for t in [srv.submit(*q) for q in qs]]
    for q, g in zip(qs, got):
        assert g["status"] == K.KDSS_OK and g["t_used"] == q[4]
        assert g["rho_prime"] <= g["upper_bound"] * (1 + 1e-12)
        a = K.kdss_solve(*q)
        if a["density"] > 0:
            assert g["density"] >= 0.99 * a["density"]
    with pytest.raises(K.KdssError) as e:
        K.Server(precision=K.KDSS_FP32K, flags=K.KDSS_FLAG_ASYNC)
    assert e.value.code == K.KDSS_ERR_INVALID_ARG
