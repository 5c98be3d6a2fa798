"""Pins of the oracle's CPSample (Sec. 5, Alg. 4) against definitions
computed independently here: the greedy colouring against networkx, the
k-color path counts and the cliques among the paths against brute-force
enumeration, every sample against the path of its rank in the enumeration
order (readings S1-S3 of kdss_oracle.c), and the whole algorithm against the
paper's example."""
import networkx as nx
import numpy as np
import pytest

import oracle as O
import synth

MASK = (1 << 64) - 1


def _splitmix(seed, index):
    z = (seed + (index + 1) * 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def _prep(n, s, d):
    off, adj = O.csr(n, s, d)
    core, rnd, dg = O.peel(n, off, adj)
    rank, _ = O.order(n, core, rnd)
    return off, adj, rank, dg


def _paths(n, off, adj, color, k):
    """All increasing-colour paths of k vertices, in the order start id, then
    each next vertex in adjacency order."""
    out = []

    def walk(path):
        if len(path) == k:
            out.append(tuple(path))
            return
        v = path[-1]
        for e in range(off[v], off[v + 1]):
            w = int(adj[e])
            if color[w] > color[v]:
                walk(path + [w])

    for v in range(n):
        walk([v])
    return out


GRAPHS = [synth.g1(), synth.erdos_renyi(40, 0.3, 5), synth.erdos_renyi(60, 0.15, 6),
          synth.chung_lu(200, 8.0, 2.4, 7, plant_size=10, plant_prob=0.9)[:3]]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_greedy_colouring_is_networkx_greedy_in_the_same_order(gi):
    n, s, d = GRAPHS[gi]
    off, adj, rank, dg = _prep(n, s, d)
    color, ncol = O.color_greedy(n, off, adj, rank)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((int(a), int(b)) for a, b in zip(s, d) if a != b)
    order = sorted(range(n), key=lambda v: -int(rank[v]))
    want = nx.greedy_color(G, strategy=lambda g, c: iter(order))
    assert [want[v] for v in range(n)] == color.tolist()
    assert all(color[a] != color[b] for a, b in G.edges())
    assert ncol == color.max() + 1 <= dg + 1       # a degeneracy order needs at most dg + 1


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("k", [2, 3, 4])
def test_color_path_counts_and_their_cliques(gi, k):
    n, s, d = GRAPHS[gi]
    off, adj, rank, _ = _prep(n, s, d)
    color, _ = O.color_greedy(n, off, adj, rank)
    dp = O.ccpath_dp(n, off, adj, color, k)
    for i in range(1, k + 1):
        paths = _paths(n, off, adj, color, i)
        per_start = np.bincount([p[0] for p in paths], minlength=n) if paths else np.zeros(n)
        assert dp[:, i - 1].tolist() == per_start.tolist()
    adjset = {(int(a), int(b)) for a, b in zip(s, d)} | {(int(b), int(a)) for a, b in zip(s, d)}
    cl_paths = sorted(tuple(sorted(p)) for p in _paths(n, off, adj, color, k)
                      if all((p[a], p[b]) in adjset for a in range(k) for b in range(a + 1, k)))
    want = sorted(tuple(int(x) for x in row) for row in O.list_cliques(n, off, adj, k))
    assert cl_paths == want                        # every clique is exactly one path (S2)


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_each_sample_is_the_path_of_its_rank(gi):
    n, s, d = GRAPHS[gi]
    k, t, seed = 3, 300, 12345 + gi
    off, adj, rank, _ = _prep(n, s, d)
    color, _ = O.color_greedy(n, off, adj, rank)
    dp = O.ccpath_dp(n, off, adj, color, k)
    paths, flags, total = O.ccpath_sample(n, off, adj, color, k, dp, t, seed)
    allp = _paths(n, off, adj, color, k)
    assert total == len(allp)
    adjset = {(int(a), int(b)) for a, b in zip(s, d)} | {(int(b), int(a)) for a, b in zip(s, d)}
    for j in range(t):
        R = ((_splitmix(seed, j) >> 11) * total) >> 53
        assert tuple(paths[j].tolist()) == allp[R]
        p = allp[R]
        assert flags[j] == all((p[a], p[b]) in adjset for a in range(k) for b in range(a + 1, k))


def test_cpsample_finds_the_example_densest_subgraph():
    """G1 (Ex. 1.1): with enough samples every triangle is in the sample set,
    Alg. 1 over it is Alg. 1 over all triangles, and the prefix is
    {u1..u6} at density 4/3."""
    n, s, d = synth.g1()
    res = O.cpsample(n, s, d, 3, 2000, 200, 3)
    assert len(res["cliques"]) == 9
    assert res["ids"].tolist() == [1, 2, 3, 4, 5, 6]
    assert res["count"] == 8 and res["istar"] == 6
