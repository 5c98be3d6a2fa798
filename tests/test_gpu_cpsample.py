"""CPSample (Sec. 5, Alg. 4) on the GPU (kdss_cpsample) against the oracle.

Both sides colour greedily by decreasing rank, count increasing-colour
k-paths exactly, draw sample j as the path of rank floor((x_j >> 11) *
#paths / 2^53) with x_j word j of SplitMix64, keep the set of sampled
cliques, run synchronous Alg. 1 and extract the sampled-density prefix: all
integer work, so every count, the sample set's size, i*, the node set and
the bound must be equal.
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


CASES = {
    "g1_k3": lambda: (*synth.g1(), 3, 500, 50),
    "er60_k3": lambda: (*synth.erdos_renyi(60, 0.2, 31), 3, 4000, 40),
    "er120_k4": lambda: (*synth.erdos_renyi(120, 0.25, 32), 4, 20000, 30),
    "chunglu5k_k4": lambda: (*synth.chung_lu(5000, 12.0, 2.4, 33, plant_size=30, plant_prob=0.9)[:3], 4, 30000, 30),
    "rmat2k_k5": lambda: (*synth.batch_rmat_graph(7, 2000), 5, 20000, 30),
    "er200_k2": lambda: (*synth.erdos_renyi(200, 0.05, 34), 2, 3000, 60),
    "no_samples": lambda: (*synth.erdos_renyi(50, 0.2, 35), 3, 0, 10),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_cpsample_matches_the_oracle(name):
    n, s, d, k, t, T = CASES[name]()
    seed = 0x5EED + len(name)
    got = K.kdss_cpsample(n, s, d, k, t, T, seed)
    want = O.cpsample(n, s, d, k, t, T, seed)
    st = got["stats"]
    assert st["colors"] == want["ncolors"]
    assert st["paths_total"] == want["paths_total"]
    assert st["samples"] == t
    assert st["samples_clique"] == want["samples_clique"]
    assert st["cliques"] == len(want["cliques"])
    assert got["istar"] == want["istar"] and got["count"] == want["count"]
    assert got["ids"].tolist() == want["ids"].tolist()
    assert got["upper_bound"] == pytest.approx(want["upper_bound"], rel=1e-12, abs=1e-12)


def test_cpsample_with_enough_samples_finds_the_example_subgraph():
    n, s, d = synth.g1()
    got = K.kdss_cpsample(n, s, d, 3, 2000, 200, 3)
    assert got["stats"]["cliques"] == 9
    assert got["ids"].tolist() == [1, 2, 3, 4, 5, 6] and got["count"] == 8


def test_cpsample_rejects_bad_arguments():
    n, s, d = synth.g1()
    for k, t, T in ((1, 10, 10), (17, 10, 10), (3, -1, 10), (3, 10, -1)):
        with pytest.raises(K.KdssError) as e:
            K.kdss_cpsample(n, s, d, k, t, T, 1)
        assert e.value.code == K.KDSS_ERR_INVALID_ARG
