"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Nothing here re-derives the oracle's own formulas: every check compares the
oracle with something independent of it -- values printed in the paper for its
worked example (tests/golden/g1_example.txt), networkx, brute force over all
subsets, an explicit clique listing, or a closed-form optimality condition.
"""
from fractions import Fraction
from itertools import combinations
import random

import numpy as np
import pytest

import oracle as O
import synth
from conftest import load_golden

G = load_golden("g1_example.txt")
GI = load_golden("g1_iterations.txt")


def _pairs_from_golden(lines):
    out = []
    for ln in lines:
        a, b = ln.split("|")
        out.append((tuple(sorted(int(x) for x in a.split())),
                    tuple(sorted(int(x) for x in b.split()))))
    return sorted(out)


def _g1():
    n, s, d = synth.g1()
    edges = [tuple(int(x) for x in e.split("-")) for e in G["edges"][0].split()]
    assert sorted(map(tuple, map(sorted, zip(s.tolist(), d.tolist())))) == sorted(
        tuple(sorted(e)) for e in edges)
    return n, s, d


def _graph(n, s, d, kind=O.ORDER_PEEL):
    off, adj = O.csr(n, s, d)
    core, rnd, dg = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd, kind)
    return off, adj, core, rnd, dg, rank, vert


# ---------------------------------------------------------------------------
# The paper's worked example G1
# ---------------------------------------------------------------------------

def test_g1_triangles_and_densest_subgraph():
    """Sec. 1 Example 1.1: 9 triangles on 7 nodes; {u1..u6} at 4/3 > 9/7."""
    n, s, d = _g1()
    off, adj, *_ = _graph(n, s, d)
    cl = O.list_cliques(n, off, adj, 3)
    assert len(cl) == int(G["triangles"][0])
    masks = [sum(1 << int(v) for v in c) for c in cl]
    bm, num, den, union = O.brute_best(n, masks, [1] * len(masks))
    want = [int(x) for x in G["densest"][0].split()]
    assert bm == sum(1 << v for v in want) and union == bm
    assert Fraction(num, den) == Fraction(G["densest_density"][0])
    assert Fraction(len(cl), n) == Fraction(G["whole_density"][0])


def test_g1_sct_matches_example_2_2():
    """Example 2.2: the five SCT pairs of G1 (vertex order u0 < ... < u6)."""
    n, s, d = _g1()
    off, adj, core, rnd, dg, rank, vert = _graph(n, s, d, O.ORDER_CORE)
    assert vert.tolist() == list(range(7))
    sc = O.sct(n, off, adj, rank, vert, 3)
    assert O.canonical_pairs(sc) == _pairs_from_golden(G["pair"])


def test_g1_example_3_1_pbupdate_steps():
    """Example 3.1: P4 then P3 from r = 0 (the remainder step, then a whole
    round of Alg. 3)."""
    r = np.zeros(7, np.uint64)
    for step in ("ex31_step1", "ex31_step2"):
        (hold, piv), = _pairs_from_golden(G[step + "_pair"])
        ids = np.array(list(hold) + list(piv), np.int32)
        delta = O.pbupdate_alg3(ids, r[ids], len(hold), 3)
        got = {int(i): int(x) for i, x in zip(ids, delta) if x}
        want = dict(tuple(map(int, t.split(":"))) for t in G[step + "_delta"][0].split())
        assert got == want
        r[ids] += delta


def test_g1_psctl_extracts_densest():
    """Alg. 2 on G1 returns {u1..u6} with 8 triangles (density 4/3)."""
    n, s, d = _g1()
    for kind in (O.ORDER_PEEL, O.ORDER_CORE):
        res = O.solve(n, s, d, 3, 100, order_kind=kind)
        assert res["istar"] == 6
        assert res["ids"].tolist() == [int(x) for x in G["densest"][0].split()]
        assert res["count"] == int(G["densest_count"][0])
        assert res["c_k"] == int(G["triangles"][0])


def test_g1_converges_to_sct_cp_optimum():
    """r_T / T tends to the SCT-CP optimum r* = (1, 4/3 x 6) of G1: the
    first batch H(r*) = {u1..u6} at rho_3 = 4/3 (Lemma 2.3 / Thm 3.3), and u0
    keeps the one triangle it cannot hand to a denser node."""
    n, s, d = _g1()
    off, adj, core, rnd, dg, rank, vert = _graph(n, s, d, O.ORDER_CORE)
    sc = O.sct(n, off, adj, rank, vert, 3)
    T = 3000
    r = O.fw_sync(n, sc, 3, T) / T
    assert abs(r[0] - 1.0) < 1e-3
    assert np.all(np.abs(r[1:] - 4.0 / 3.0) < 1e-3)


def _g1_pairs_in_listed_order():
    """The five pairs of Example 2.2 as arrays, in the order listed there,
    hold nodes first (the oracle's pair layout)."""
    po, nodes, h = [0], [], []
    for ln in G["pair"]:
        a, b = ln.split("|")
        hold, piv = [int(x) for x in a.split()], [int(x) for x in b.split()]
        nodes += hold + piv
        h.append(len(hold))
        po.append(len(nodes))
    return {"pair_off": np.array(po, np.int64), "nodes": np.array(nodes, np.int32),
            "h": np.array(h, np.int32)}


def test_g1_inplace_iterations_match_hand_trace():
    """Alg. 2 as printed (each pair reads r as the pairs before it in the
    same iteration left it), Alg. 3 with the remainder to the lowest ids: the
    first two iterations on G1 equal the trace derived by hand in
    tests/golden/g1_iterations.txt, which differs from the synchronous form
    already at t = 1."""
    sc = _g1_pairs_in_listed_order()
    for t, key in ((1, "seq_r1"), (2, "seq_r2")):
        want = [int(x) for x in GI[key][0].split()]
        assert O.fw_seq(7, sc, 3, t).tolist() == want
    assert O.fw_sync(7, sc, 3, 1).tolist() != [int(x) for x in GI["seq_r1"][0].split()]


def test_g1_continuous_iterations_match_hand_trace():
    """Synchronous iterations of the continuous water-filling rule (reading
    R11 of the FP32 path): r_1 and r_2 on G1 equal the exact fractions
    derived by hand in tests/golden/g1_iterations.txt."""
    sc = _g1_pairs_in_listed_order()
    for t, key in ((1, "cont_r1"), (2, "cont_r2")):
        want = np.array([float(Fraction(x)) for x in GI[key][0].split()])
        got = O.fw_cont(7, sc, 3, t)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(want)


def test_g1_continuous_rule_converges_to_sct_cp_optimum():
    """The continuous rule reaches the same SCT-CP optimum of G1 as the
    integer rule: r_T / T -> r* = (1, 4/3 x 6)."""
    n, s, d = _g1()
    off, adj, core, rnd, dg, rank, vert = _graph(n, s, d, O.ORDER_CORE)
    sc = O.sct(n, off, adj, rank, vert, 3)
    T = 3000
    r = O.fw_cont(n, sc, 3, T) / T
    assert abs(r[0] - 1.0) < 1e-3
    assert np.all(np.abs(r[1:] - 4.0 / 3.0) < 1e-3)


# ---------------------------------------------------------------------------
# A1-A2 against networkx
# ---------------------------------------------------------------------------

def test_csr_and_core_numbers_against_networkx():
    nx = pytest.importorskip("networkx")
    for seed in range(5):
        n, s, d, _ = synth.chung_lu(400, 8.0, 2.3, seed, plant_size=15, plant_prob=0.8)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
        Gx = nx.Graph()
        Gx.add_nodes_from(range(n))
        Gx.add_edges_from((int(a), int(b)) for a, b in zip(s, d) if a != b)
        assert len(adj) == 2 * Gx.number_of_edges()
        for v in range(n):
            assert adj[off[v]:off[v + 1]].tolist() == sorted(Gx.neighbors(v))
        cn = nx.core_number(Gx)
        assert [cn[v] for v in range(n)] == core.tolist()
        assert dg == max(cn.values())
        # every vertex has at most core(v) later neighbours in the peel order
        for v in range(n):
            later = np.sum(rank[adj[off[v]:off[v + 1]]] > rank[v])
            assert later <= core[v]


def test_peel_rounds_satisfy_their_definition():
    """The rounds of the peeling that orders the SCT build (Sec. 2's
    degeneracy; the key (round, id) of the vertex order).  The rounds are
    checked against the conditions that fix them, not recomputed: round r at
    level L removes exactly the present vertices with at most L present
    neighbours, and L rises, to the smallest present degree, only when no
    present vertex is at or below it; every vertex is removed."""
    for seed in range(4):
        n, s, d, _ = synth.chung_lu(300, 8.0, 2.3, 40 + seed, plant_size=12, plant_prob=0.8)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
        alive = np.ones(n, bool)
        level = 0
        for r in range(int(rnd.max()) + 1):
            deg = np.array([int(alive[adj[off[v]:off[v + 1]]].sum()) for v in range(n)])
            take = rnd == r
            levels = set(core[take].tolist())
            assert len(levels) == 1, (seed, r)
            lr = levels.pop()
            assert lr == max(level, int(deg[alive].min()))
            assert np.array_equal(take, alive & (deg <= lr)), (seed, r)
            alive &= ~take
            level = lr
        assert not alive.any() and dg == level


# ---------------------------------------------------------------------------
# The SCT against the explicit clique list (Lemmas 2.4-2.6)
# ---------------------------------------------------------------------------

def _expand(sc, k):
    """All k-cliques encoded by the pairs (Lemma 2.5)."""
    out = []
    po, nodes, h = sc["pair_off"], sc["nodes"], sc["h"]
    for q in range(len(h)):
        seg = nodes[po[q]:po[q + 1]].tolist()
        hold, piv = seg[:h[q]], seg[h[q]:]
        for extra in combinations(piv, k - len(hold)):
            out.append(tuple(sorted(hold + list(extra))))
    return out


@pytest.mark.parametrize("kind", [O.ORDER_PEEL, O.ORDER_CORE])
def test_sct_partitions_the_k_cliques(kind):
    rng = random.Random(7)
    for trial in range(12):
        n = rng.randint(15, 45)
        p = rng.uniform(0.15, 0.5)
        n, s, d = synth.erdos_renyi(n, p, 100 + trial)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d, kind)
        adjset = {(int(a), int(b)) for a, b in zip(np.repeat(np.arange(n), np.diff(off)), adj)}
        for k in (2, 3, 4, 5):
            sc = O.sct(n, off, adj, rank, vert, k)
            listed = sorted(map(tuple, O.list_cliques(n, off, adj, k).tolist()))
            enc = _expand(sc, k)
            assert len(enc) == len(set(enc)), "pairs overlap"          # disjoint
            assert sorted(enc) == listed                               # cover
            po, nodes, h = sc["pair_off"], sc["nodes"], sc["h"]
            total_cap = 0
            for q in range(len(h)):
                seg = nodes[po[q]:po[q + 1]].tolist()
                hh, pp = h[q], len(seg) - h[q]
                assert hh <= k <= len(seg)                             # Lemma 2.5
                assert all((a, b) in adjset for a, b in combinations(seg, 2))  # V(P) clique
                # Lemma 2.6 per node, counted on the expanded cliques
                cl_p = [set(seg[:hh]) | set(e) for e in combinations(seg[hh:], k - hh)]
                for i, u in enumerate(seg):
                    cnt = sum(1 for c in cl_p if u in c)
                    cap = O.binom(pp, k - hh) if i < hh else O.binom(pp - 1, k - hh - 1)
                    assert cnt == cap
                    total_cap += cap
            assert total_cap == k * len(listed)                        # sum of caps = k c_k


# ---------------------------------------------------------------------------
# PBUpdate: Alg. 3, one-clique-at-a-time greedy and the closed-form level
# ---------------------------------------------------------------------------

def _random_pair(rng):
    k = rng.randint(2, 7)
    h = rng.randint(1, k)
    p = rng.randint(max(0, k - h), 9)
    ln = h + p
    ids = rng.sample(range(1000), ln)
    spread = rng.choice([0, 1, 2, 5, 50, 10 ** 6])
    r = [rng.randint(0, spread) for _ in range(ln)]
    if rng.random() < 0.3:
        r = [x - x % 3 for x in r]   # many ties
    return np.array(ids, np.int32), np.array(r, np.uint64), h, k


def test_pbupdate_three_restatements_agree():
    """Alg. 3 (with reading R6) equals the per-clique greedy and the closed
    form of the water level on 20,000 random pairs."""
    rng = random.Random(11)
    for _ in range(20000):
        ids, r, h, k = _random_pair(rng)
        a = O.pbupdate_alg3(ids, r, h, k)
        b = O.pbupdate_greedy(ids, r, h, k)
        c = O.pbupdate_level(ids, r, h, k)
        assert a.tolist() == b.tolist() == c.tolist()


def test_pbupdate_is_an_optimal_integer_allocation():
    """KKT check of an allocation minimising the sum of squares under C3-C4:
    all n_C units are placed, caps hold, and no unit can move from a node to
    a node with spare capacity that ends lower by 2 or more."""
    rng = random.Random(12)
    for _ in range(5000):
        ids, r, h, k = _random_pair(rng)
        ln, p = len(ids), len(ids) - h
        nC = O.binom(p, k - h)
        cap = [O.binom(p, k - h)] * h + [O.binom(p - 1, k - h - 1)] * p
        dl = O.pbupdate_alg3(ids, r, h, k).astype(object)
        assert sum(dl) == nC
        fin = [int(r[i]) + int(dl[i]) for i in range(ln)]
        for i in range(ln):
            assert 0 <= dl[i] <= cap[i]
            if dl[i] == 0:
                continue
            for j in range(ln):
                if dl[j] < cap[j]:
                    assert fin[i] - 1 <= fin[j]


def test_binomials_beyond_64_bits():
    """The 128-bit binomials equal exact integer arithmetic (math.comb) where
    64 bits overflow, and a value beyond 128 bits is refused."""
    import math
    for a, b in [(70, 35), (100, 39), (120, 39), (127, 63), (200, 30), (64, 32)]:
        assert O.binom128(a, b) == math.comb(a, b)
    with pytest.raises(OverflowError):
        O.binom128(300, 150)
    with pytest.raises(OverflowError):
        O.binom(100, 39)


def test_pbupdate_continuous_with_counts_beyond_64_bits():
    """The continuous water level of a pair whose n_C = C(p, k - h) needs
    more than 64 bits: all n_C units are placed (to double rounding), no node
    exceeds its Lemma 2.6 cap, and the receiving nodes share one level."""
    import math
    rng = random.Random(17)
    for _ in range(200):
        p = rng.randint(90, 130)
        h = rng.randint(1, 3)
        k = h + rng.randint(30, 45)
        ids = np.array(rng.sample(range(5000), h + p), np.int32)
        nC = math.comb(p, k - h)
        assert nC >= 2 ** 64
        r = np.array([rng.random() * nC * 3 for _ in ids])
        dl = O.pbupdate_cont(ids, r, h, k)
        cap = [float(nC)] * h + [float(math.comb(p - 1, k - h - 1))] * p
        assert abs(dl.sum() - nC) <= 1e-9 * nC
        assert all(-1e-9 * nC <= dl[i] <= cap[i] * (1 + 1e-12) for i in range(len(ids)))
        fin = r + dl
        recv = [i for i in range(len(ids)) if dl[i] > 1e-9 * nC and dl[i] < cap[i] * (1 - 1e-9)]
        if recv:
            L = fin[recv[0]]
            assert all(abs(fin[i] - L) <= 1e-9 * L for i in recv)


def test_pbupdate_continuous_is_the_exact_water_level():
    """Continuous rule: all units placed, caps hold, and every node that
    receives weight ends at one common level L that no node with spare
    capacity lies below."""
    rng = random.Random(13)
    for _ in range(3000):
        ids, r, h, k = _random_pair(rng)
        rr = r.astype(np.float64) + np.array([rng.random() for _ in r])
        dl = O.pbupdate_cont(ids, rr, h, k)
        ln, p = len(ids), len(ids) - h
        nC = O.binom(p, k - h)
        cap = [float(O.binom(p, k - h))] * h + [float(O.binom(p - 1, k - h - 1))] * p
        assert abs(dl.sum() - nC) <= 1e-9 * max(1.0, nC)
        fin = rr + dl
        recv = [i for i in range(ln) if dl[i] > 1e-9 and dl[i] < cap[i] - 1e-9]
        if recv:
            L = fin[recv[0]]
            for i in recv:
                assert abs(fin[i] - L) <= 1e-6 * max(1.0, L)
            for j in range(ln):
                if dl[j] < cap[j] - 1e-9:
                    assert fin[j] >= L - 1e-6 * max(1.0, L)


# ---------------------------------------------------------------------------
# FW invariants (Lemma 3.1, Thms 3.5-3.6) and brute force (Def. 2.1, Thm 3.4)
# ---------------------------------------------------------------------------

def _planted(n, p, size, seed):
    n, s, d = synth.erdos_renyi(n, p, seed)
    rng = random.Random(seed)
    nodes = rng.sample(range(n), size)
    extra = [(a, b) for a, b in combinations(nodes, 2) if rng.random() < 0.9]
    s = np.concatenate([s, np.array([a for a, _ in extra], np.int32)])
    d = np.concatenate([d, np.array([b for _, b in extra], np.int32)])
    return n, s, d


def test_fw_invariants_and_weak_duality():
    """sum_u r_t(u) = t c_k and r_t(u) <= t cnt_k(u) (Lemma 3.1); the best
    rho'(V_i) never exceeds max_u r_t(u)/t (weak duality, Thms 3.5-3.6); the
    extracted rho_k never exceeds the Alg. 1 bound max_u r^CP_t(u)/t."""
    for seed in range(4):
        n, s, d = _planted(40, 0.15, 10, 50 + seed)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
        for k in (3, 4):
            sc = O.sct(n, off, adj, rank, vert, k)
            cl = O.list_cliques(n, off, adj, k)
            ck = len(cl)
            cnt = np.bincount(cl.reshape(-1), minlength=n) if ck else np.zeros(n, int)
            rcp = O.fw_cliques(n, cl, k, 50)
            for t in (1, 2, 3, 7, 20):
                r = O.fw_sync(n, sc, k, t)
                assert int(r.astype(object).sum()) == t * ck
                assert np.all(r.astype(np.int64) <= t * cnt)
                ordr = O.sort_desc(r)
                lo, hi, flo, fhi = O.prefix_counts_pairs(n, ordr, sc, k)
                best_rp = max(Fraction(int(flo[i]), i) for i in range(1, n + 1))
                assert best_rp <= Fraction(int(r.max()), t)
                i = O.argmax_density(lo, hi)
                assert Fraction(int(lo[i]), i) <= Fraction(int(rcp.max()), 50)


def test_fw_cont_and_fw_seq_invariants_and_weak_duality():
    """Lemma 3.1 and Thms 3.5-3.6 for the continuous rule (synchronous) and
    for the in-place integer iterations: sum_u r_t(u) = t c_k (to 1e-9
    relative in FP64, exactly for the integers), r_t(u) <= t cnt_k(u) with
    cnt_k(u) from the explicit clique list, and max_u r_t(u)/t >= the best
    rho'(S) over all subsets S (brute force) at every t."""
    for seed in range(4):
        n, s, d = _planted(13 + seed % 2, 0.25, 6, 700 + seed)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
        for k in (3, 4):
            sc = O.sct(n, off, adj, rank, vert, k)
            cl = O.list_cliques(n, off, adj, k)
            ck = len(cl)
            if ck == 0:
                continue
            cnt = np.bincount(cl.reshape(-1), minlength=n)
            pm, ph = sc["pair_off"], sc["h"]
            pmasks, pw = [], []
            for q in range(len(ph)):
                seg = sc["nodes"][pm[q]:pm[q + 1]]
                pmasks.append(sum(1 << int(v) for v in seg))
                pw.append(O.binom(len(seg) - ph[q], k - ph[q]))
            _, pn, pd, _ = O.brute_best(n, pmasks, pw)
            rho_p = Fraction(pn, pd)
            for t in (1, 2, 3, 6, 25):
                rc = O.fw_cont(n, sc, k, t)
                assert abs(rc.sum() - t * ck) <= 1e-9 * t * ck
                assert np.all(rc <= t * cnt * (1 + 1e-12) + 1e-9)
                assert rc.max() / t >= float(rho_p) * (1 - 1e-12)
                rs = O.fw_seq(n, sc, k, t)
                assert int(rs.astype(object).sum()) == t * ck
                assert np.all(rs.astype(np.int64) <= t * cnt)
                assert Fraction(int(rs.max()), t) >= rho_p
            # both reach the SCT-CP bound: max r / T tends to max rho'(S)
            T = 3000
            assert float(O.fw_cont(n, sc, k, T).max()) / T <= float(rho_p) * 1.02 + 1e-9
            assert float(O.fw_seq(n, sc, k, T).max()) / T <= float(rho_p) * 1.02 + 1e-9


def test_continuous_trajectory_amplifies_rounding_but_not_the_subgraph():
    """The FW iterates of the continuous rule (Alg. 2 with the water level of
    Sec. 3.2 taken exactly, gamma_t = 1/t) are sensitive to their input: in
    FP64, a relative change of 1e-13 on the 50 largest entries of r_50 grows
    by more than 1e3 within 10 iterations and to more than 1e-3 of max r
    after 40, while both runs keep sum r_t = t c_k (Lemma 3.1) and extract the
    same densest prefix (Alg. 2's final sort and prefix step).  So r at T
    cannot be compared across implementations that round differently at a
    tolerance like 1e-5; the comparison that holds is per iteration, from the
    same state, plus the extracted subgraph and the invariants at T."""
    n, s, d = synth.chung_lu(3000, 12.0, 2.4, 9, plant_size=25, plant_prob=0.85)[:3]
    k = 4
    off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
    sc = O.sct(n, off, adj, rank, vert, k)
    pm, ph = sc["pair_off"], sc["h"]
    ck = sum(O.binom(int(pm[q + 1] - pm[q] - ph[q]), k - int(ph[q])) for q in range(len(ph)))
    ra = O.fw_cont(n, sc, k, 50)
    rb = ra.copy()
    top = np.argsort(-ra)[:50]
    rb[top] *= 1.0 + 1e-13 * np.random.default_rng(1).standard_normal(top.size)
    rel = lambda x, y: float(np.abs(x - y).max() / np.abs(x).max())
    d0 = rel(ra, rb)
    assert 0 < d0 < 1e-12
    xa, xb = O.fw_cont(n, sc, k, 10, r0=ra), O.fw_cont(n, sc, k, 10, r0=rb)
    assert rel(xa, xb) > 1e3 * d0
    xa, xb = O.fw_cont(n, sc, k, 30, r0=xa), O.fw_cont(n, sc, k, 30, r0=xb)
    assert rel(xa, xb) > 1e-3
    # splitting the iterations over calls changes nothing: the growth comes
    # from the perturbation alone
    assert np.array_equal(xa, O.fw_cont(n, sc, k, 90))
    found = []
    for x in (xa, xb):
        assert abs(x.sum() - 90 * ck) <= 1e-12 * 90 * ck
        od = O.sort_desc(x)
        lo, hi, _, _ = O.prefix_counts_pairs(n, od, sc, k)
        i = O.argmax_density(lo, hi)
        found.append((i, int(lo[i]), sorted(od[:i].tolist())))
    assert found[0] == found[1] and found[0][0] > 0


def test_fw_seq_equals_synchronous_on_node_disjoint_pairs():
    """When no two pairs share a node, no pair can see another's update, so
    the in-place and synchronous iterations coincide (integer rule)."""
    rng = random.Random(21)
    po, nodes, h = [0], [], []
    nxt = 0
    for _ in range(40):
        ln = rng.randint(3, 9)
        hh = rng.randint(1, 3)
        nodes += list(range(nxt, nxt + ln))
        nxt += ln
        h.append(hh)
        po.append(len(nodes))
    sc = {"pair_off": np.array(po, np.int64), "nodes": np.array(nodes, np.int32),
          "h": np.array(h, np.int32)}
    for k in (3, 4):
        ok = [q for q in range(len(h)) if h[q] <= k <= po[q + 1] - po[q]]
        sub = {"pair_off": np.array([0] + list(np.cumsum([po[q + 1] - po[q] for q in ok])),
                                    np.int64),
               "nodes": np.concatenate([sc["nodes"][po[q]:po[q + 1]] for q in ok]),
               "h": np.array([h[q] for q in ok], np.int32)}
        r0 = np.array([rng.randint(0, 5) for _ in range(nxt)], np.uint64)
        assert np.array_equal(O.fw_seq(nxt, sub, k, 9, r0), O.fw_sync(nxt, sub, k, 9, r0))


def test_prefix_counts_from_pairs_equal_explicit_list():
    """C_k(V_i) from the SCT pairs (Lemma 2.5-2.6) equals the explicit count."""
    rng = np.random.default_rng(3)
    for seed in range(5):
        n, s, d = _planted(50, 0.12, 12, 80 + seed)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
        for k in (2, 3, 5):
            sc = O.sct(n, off, adj, rank, vert, k)
            cl = O.list_cliques(n, off, adj, k)
            ordr = rng.permutation(n).astype(np.int32)
            a, ah = O.prefix_counts_cliques(n, ordr, cl, k)
            b, bh, _, _ = O.prefix_counts_pairs(n, ordr, sc, k)
            assert a.tolist() == b.tolist() and ah.tolist() == bh.tolist()


def test_rho_prime_prefix_counts_equal_their_definition():
    """F_i, the numerator of rho'(V_i) (Thm 3.6: the cliques of the pairs P
    whose node set V(P) lies inside V_i, n_C = C(|V_p|, k - |V_h|) each, Lemma
    2.6), equals a direct count over the pairs for every prefix of a random
    order; a pair enters once its last node does."""
    rng = np.random.default_rng(5)
    for seed in range(4):
        n, s, d = _planted(40, 0.15, 10, 120 + seed)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
        for k in (3, 4):
            sc = O.sct(n, off, adj, rank, vert, k)
            pm, ph, nodes = sc["pair_off"], sc["h"], sc["nodes"]
            ordr = rng.permutation(n).astype(np.int32)
            pos = np.empty(n, np.int64)
            pos[ordr] = np.arange(n)
            want = [0] * (n + 1)
            for q in range(len(ph)):
                seg = nodes[pm[q]:pm[q + 1]]
                enter = int(pos[seg].max()) + 1          # V(P) inside V_i from i = enter on
                nc = O.binom(len(seg) - int(ph[q]), k - int(ph[q]))
                for i in range(enter, n + 1):
                    want[i] += nc
            _, _, flo, fhi = O.prefix_counts_pairs(n, ordr, sc, k)
            got = [int(a) | (int(b) << 64) for a, b in zip(flo, fhi)]
            assert got == want


def test_final_sort_is_r_descending_with_ties_to_ascending_ids():
    """The node order of the extraction (Alg. 2's final sort; reading R4 for
    ties) against numpy's lexicographic sort on the keys (-r, id), for
    integer and FP64 r with many ties."""
    rng = np.random.default_rng(11)
    for n in (1, 2, 7, 300, 2000):
        ru = rng.integers(0, 6, n).astype(np.uint64) * np.uint64(1 << 40)
        want = np.lexsort((np.arange(n), -ru.astype(np.float64)))
        assert O.sort_desc(ru).tolist() == want.tolist()
        rf = rng.integers(0, 6, n).astype(np.float64) / 3.0
        want = np.lexsort((np.arange(n), -rf))
        assert O.sort_desc(rf).tolist() == want.tolist()


def test_argmax_takes_the_largest_prefix_on_ties():
    lo = np.array([0, 1, 2, 3, 3, 5, 6], np.uint64)   # 1/1 = 2/2 = 3/3 = 6/6
    hi = np.zeros(7, np.uint64)
    assert O.argmax_density(lo, hi) == 6
    lo = np.array([0, 0, 3, 3, 4], np.uint64)          # 3/2 > 3/3, 4/4
    assert O.argmax_density(lo, np.zeros(5, np.uint64)) == 2


@pytest.mark.parametrize("k", [2, 3, 4])
def test_brute_force_small_graphs(k):
    """n <= 14: the k-clique densest subgraph V* (Def. 2.1, maximal on ties)
    by enumeration of all subsets; PSCTL after many iterations meets the
    bound of Thm 3.4 and max_u r/T tends to max_S rho'(S) (Thms 3.5-3.6);
    Alg. 1 (CP(G), Lemma 2.3) extracts V* itself."""
    for seed in range(6):
        n, s, d = _planted(12 + seed % 3, 0.25, 6, 200 + seed + 10 * k)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
        cl = O.list_cliques(n, off, adj, k)
        if len(cl) == 0:
            continue
        masks = [sum(1 << int(v) for v in c) for c in cl]
        bm, num, den, union = O.brute_best(n, masks, [1] * len(masks))
        assert union == bm                      # the maximal V* contains all maximisers
        rho_star = Fraction(num, den)
        sc = O.sct(n, off, adj, rank, vert, k)
        pm, ph = sc["pair_off"], sc["h"]
        pmasks, pw = [], []
        for q in range(len(ph)):
            seg = sc["nodes"][pm[q]:pm[q + 1]]
            pmasks.append(sum(1 << int(v) for v in seg))
            pw.append(O.binom(len(seg) - ph[q], k - ph[q]))
        _, pn, pd, _ = O.brute_best(n, pmasks, pw)
        rho_p = Fraction(pn, pd)
        assert rho_p <= rho_star                # rho'(S) <= rho_k(S)
        T = 4000
        res_r = O.fw_sync(n, sc, k, T)
        ordr = O.sort_desc(res_r)
        lo, hi, _, _ = O.prefix_counts_pairs(n, ordr, sc, k)
        i = O.argmax_density(lo, hi)
        got = Fraction(int(lo[i]), i)
        assert got > rho_star * (1 - Fraction(1, k * den))                # Thm 3.4
        ub = Fraction(int(res_r.max()), T)
        assert ub >= rho_p and float(ub) <= float(rho_p) * 1.02 + 1e-9     # Thm 3.5-3.6
        rcp = O.fw_cliques(n, cl, k, T)
        o2 = O.sort_desc(rcp)
        lo2, hi2 = O.prefix_counts_cliques(n, o2, cl, k)
        i2 = O.argmax_density(lo2, hi2)
        assert sorted(o2[:i2].tolist()) == [v for v in range(n) if bm >> v & 1]


def test_sequential_and_synchronous_reach_the_same_density():
    """Both readings of Alg. 2's pair loop reach the paper's density on G1."""
    n, s, d = _g1()
    a = O.solve(n, s, d, 3, 50, mode="seq")
    b = O.solve(n, s, d, 3, 50, mode="sync")
    assert a["istar"] == b["istar"] == 6 and a["count"] == b["count"] == 8


def test_threaded_synchronous_iterations_equal_the_serial_ones():
    """The host-threaded form of the synchronous iterations (the timed CPU
    baseline on all cores) sums the same integer allocations: r_T is equal."""
    for n, s, d, k, T in [(*synth.g1(), 3, 30),
                          (*synth.erdos_renyi(400, 0.04, 11), 3, 25),
                          (*synth.chung_lu(3000, 10.0, 2.4, 12, plant_size=20, plant_prob=0.9)[:3], 4, 20)]:
        off, adj = O.csr(n, s, d)
        core, rnd, _ = O.peel(n, off, adj)
        rank, vert = O.order(n, core, rnd)
        sc = O.sct(n, off, adj, rank, vert, k)
        want = O.fw_sync(n, sc, k, T)
        for th in (1, 3, 8):
            assert np.array_equal(O.fw_sync_par(n, sc, k, T, th), want)


def test_threaded_continuous_iterations_equal_the_serial_ones():
    """The host-threaded continuous-rule iterations (used to state the FP32
    path's error against FP64 on large graphs) add the same numbers in the
    same order as the serial form: r_T is bit for bit equal."""
    for n, s, d, k, T in [(*synth.g1(), 3, 40),
                          (*synth.chung_lu(3000, 10.0, 2.4, 12, plant_size=20, plant_prob=0.9)[:3], 4, 15)]:
        off, adj = O.csr(n, s, d)
        core, rnd, _ = O.peel(n, off, adj)
        rank, vert = O.order(n, core, rnd)
        sc = O.sct(n, off, adj, rank, vert, k)
        want = O.fw_cont(n, sc, k, T)
        for th in (1, 3, 8):
            assert np.array_equal(O.fw_cont_par(n, sc, k, T, th), want)


def test_alg1_synchronous_over_explicit_cliques():
    """Alg. 1 over the explicit clique list, synchronous reading: the first
    iteration from r = 0 gives every clique's unit to its lowest id (closed
    form); sum r_t = t c exactly; on vertex-disjoint cliques it equals the
    sequential form (no clique sees another's update); r_T / T is feasible
    for CP(G), so max r_T / T >= rho_k(V*) (brute force), and the prefix
    extracted from it reaches V* on small graphs (Lemma 2.3)."""
    n, s, d = synth.g1()
    off, adj = O.csr(n, s, d)
    cl = O.list_cliques(n, off, adj, 3)
    r1 = O.fw_cliques_sync(n, cl, 3, 1)
    assert r1.tolist() == np.bincount(cl.min(axis=1), minlength=n).tolist()
    rT = O.fw_cliques_sync(n, cl, 3, 57)
    assert int(rT.sum()) == 57 * len(cl)
    # disjoint triangles: synchronous == sequential
    tri = np.array([[3 * i, 3 * i + 1, 3 * i + 2] for i in range(5)], np.int32)
    assert np.array_equal(O.fw_cliques_sync(15, tri, 3, 20), O.fw_cliques(15, tri, 3, 20))
    for seed in range(4):
        n, s, d = _planted(12 + seed % 3, 0.25, 6, 500 + seed)
        off, adj, core, rnd, dg, rank, vert = _graph(n, s, d)
        for k in (2, 3):
            cl = O.list_cliques(n, off, adj, k)
            if len(cl) == 0:
                continue
            masks = [sum(1 << int(v) for v in c) for c in cl]
            bm, num, den, union = O.brute_best(n, masks, [1] * len(masks))
            T = 3000
            r = O.fw_cliques_sync(n, cl, k, T)
            assert Fraction(int(r.max()), T) >= Fraction(num, den)
            o2 = O.sort_desc(r)
            lo2, hi2 = O.prefix_counts_cliques(n, o2, cl, k)
            i2 = O.argmax_density(lo2, hi2)
            assert Fraction(int(lo2[i2]), i2) == Fraction(num, den)
