"""kdss_solve_batch: many (graph, k, T) queries solved together.

The batch joins the graphs of equal (k, T) into one disjoint union, iterates
all groups together and extracts every query from one segmented sort and
scan.  Each query's result must equal what kdss_solve returns for it alone --
bit for bit for the integer rule (INT64 and FP64 storage): the vertex order,
the SCT and r of a component of a disjoint union are those of the component
alone (peeling never crosses components).  The FP32 rule is checked against
the FP64 oracle's density within 1% and the invariants that bound it.
Invalid queries fail alone and leave the other queries' results intact.
"""
import numpy as np
import pytest

import oracle as O
import paper_2403_05775_gb300 as K
import synth

pytestmark = pytest.mark.gpu

FIELDS = ("istar", "count", "density", "upper_bound", "rho_prime", "gap", "T", "t_used", "status")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)


def _same(a, b):
    for f in FIELDS:
        assert a[f] == b[f], (f, a[f], b[f])
    assert a["ids"].tolist() == b["ids"].tolist()


def _mixed_queries():
    qs = []
    n, s, d = synth.g1()
    qs.append((n, s, d, 3, 40))
    for i, (nn, p) in enumerate([(300, 0.05), (120, 0.2), (800, 0.02)]):
        n, s, d = synth.erdos_renyi(nn, p, 30 + i)
        qs.append((n, s, d, 3 + i, 40 if i != 1 else 25))
    n, s, d, _ = synth.chung_lu(3000, 12.0, 2.4, 9, plant_size=25, plant_prob=0.85)
    qs.append((n, s, d, 4, 40))
    qs.append((n, s, d, 5, 40))
    n, s, d = synth.batch_rmat_graph(0, 2000)
    qs.append((n, s, d, 3, 40))                   # same (k, T) as g1: one union
    qs.append((0, np.zeros(0, np.int32), np.zeros(0, np.int32), 3, 40))   # empty graph
    qs.append((9, np.array([1, 2], np.int32), np.array([1, 2], np.int32), 3, 40))  # no edge left
    qs.append((60, *synth.erdos_renyi(60, 0.01, 5)[1:], 6, 40))            # no 6-clique
    qs.append((7, *synth.g1()[1:], 3, 0))        # T = 0
    return qs


@pytest.mark.parametrize("prec", [K.KDSS_INT64, K.KDSS_FP64])
def test_batch_equals_each_query_alone(prec):
    qs = _mixed_queries()
    opts = K.make_opts(precision=prec)
    got = K.kdss_solve_batch(qs, opts)
    assert len(got) == len(qs)
    for q, g in zip(qs, got):
        _same(g, K.kdss_solve(*q, opts))


def test_batch_matches_the_oracle_directly():
    qs = _mixed_queries()[:6]
    got = K.kdss_solve_batch(qs)
    for (n, s, d, k, T), g in zip(qs, got):
        o = O.solve(n, s, d, k, T)
        assert (g["istar"], g["count"], g["ids"].tolist()) == (o["istar"], o["count"], o["ids"].tolist())
        assert abs(g["upper_bound"] - o["upper_bound"]) <= 1e-12 * max(1.0, o["upper_bound"])


def test_batch_of_rmat_instances_with_mixed_k():
    """The batched R-MAT workload's shape (edge factor 16, planted 30-node
    clique, k in {3..8}) at smaller node counts: several instances per k."""
    ns, ks = synth.batch_rmat_specs(24, nmin=1e3, nmax=2e4)
    qs = []
    for i, (n, k) in enumerate(zip(ns, ks)):
        n, s, d = synth.batch_rmat_graph(i, int(n))
        qs.append((n, s, d, int(k), 30))
    got = K.kdss_solve_batch(qs)
    assert all(g["status"] == K.KDSS_OK for g in got)
    for q, g in zip(qs, got):
        _same(g, K.kdss_solve(*q))


def test_batch_fp32_density_within_one_percent_of_the_oracle():
    qs = []
    for i, (n, k) in enumerate(zip(*synth.batch_rmat_specs(8, nmin=1e3, nmax=2.5e3))):
        n, s, d = synth.batch_rmat_graph(i, int(n))
        qs.append((n, s, d, int(k), 120))
    got = K.kdss_solve_batch(qs, K.make_opts(precision=K.KDSS_FP32K))
    for (n, s, d, k, T), g in zip(qs, got):
        o = O.solve(n, s, d, k, T, mode="cont")
        assert g["status"] == K.KDSS_OK and g["T"] == T
        assert abs(g["density"] - o["density"]) <= 1e-2 * o["density"]
        assert g["density"] <= g["upper_bound"] * (1 + 1e-5)      # Thm 3.5
        assert g["rho_prime"] <= g["upper_bound"] * (1 + 1e-5)
        # the subgraph's clique count is exact whatever the precision of r:
        # count the k-cliques of the induced subgraph with the oracle
        if g["istar"]:
            inside = np.zeros(n, bool)
            inside[g["ids"]] = True
            keep = inside[s] & inside[d]
            off, adj = O.csr(n, s[keep], d[keep])
            assert g["count"] == O.count_cliques(n, off, adj, k)


def test_invalid_queries_fail_alone():
    n, s, d = synth.g1()
    good = (n, s, d, 3, 20)
    bad_edge = (5, np.array([0, 7], np.int32), np.array([1, 2], np.int32), 3, 20)
    bad_k = (n, s, d, 1, 20)
    bad_T = (n, s, d, 3, -1)
    got = K.kdss_solve_batch([good, bad_edge, good, bad_k, bad_T])
    want = K.kdss_solve(*good)
    _same(got[0], want)
    _same(got[2], want)
    assert got[1]["status"] == K.KDSS_ERR_BAD_GRAPH and got[1]["istar"] == 0
    assert got[3]["status"] == K.KDSS_ERR_INVALID_ARG
    assert got[4]["status"] == K.KDSS_ERR_INVALID_ARG
    assert K.kdss_solve_batch([]) == []


def test_batch_on_device_inputs_and_a_torch_stream():
    import torch
    qs = _mixed_queries()[:6]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        dq = [(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), k, T) for n, s, d, k, T in qs]
        got = K.kdss_solve_batch(dq, K.make_opts(stream=st))
    for q, g in zip(qs, got):
        _same(g, K.kdss_solve(*q))
