"""The root-shared form of the SCT (16-bit indices into each root's
out-neighbourhood) and the first-step kernel that gathers each neighbourhood
once per tile.

On a union of disjoint 31-cliques every root holds exactly one pair (the root
and all its later clique members), so consecutive pairs come from different
roots and a tile's neighbourhoods overflow the kernel's staging area: those
tiles go to the slow kernel whole.  Mixed with ordinary graphs, r_T must equal
the oracle's bit for bit either way.
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


def _cliques(count, size):
    s, d = [], []
    for c in range(count):
        iu = np.triu_indices(size, 1)
        s.append(iu[0] + c * size)
        d.append(iu[1] + c * size)
    return count * size, np.concatenate(s).astype(np.int32), np.concatenate(d).astype(np.int32)


def _with(n, s, d, n2, s2, d2):
    return n + n2, np.concatenate([s, s2 + n]).astype(np.int32), np.concatenate([d, d2 + n]).astype(np.int32)


@pytest.mark.parametrize("k", [3, 5])
def test_rooted_first_step_with_overflowing_tiles(k):
    n, s, d = _with(*_cliques(60, 31), *synth.chung_lu(2000, 10.0, 2.4, 41, plant_size=20,
                                                       plant_prob=0.9)[:3])
    T = 15
    off, adj = O.csr(n, s, d)
    core, rnd, _ = O.peel(n, off, adj)
    rank, vert = O.order(n, core, rnd)
    want = O.fw_sync(n, O.sct(n, off, adj, rank, vert, k), k, T)
    sct = K.kdss_build_sct(n, s, d, k)
    for prec in (K.KDSS_INT64, K.KDSS_FP64):
        for flags in (K.KDSS_FLAG_ROOTED, 0):
            o = K.make_opts(precision=prec, flags=flags)
            r, _ = K.kdss_state_copy_r(K.kdss_fw_iterate(sct, None, T, o), n, prec)
            assert np.array_equal(r.astype(np.uint64), want), (prec, flags)


@pytest.mark.parametrize("name", ["er300", "chunglu3k", "rmat2k"])
def test_rooted_first_step_equals_the_oracle(name):
    graphs = {"er300": lambda: synth.erdos_renyi(300, 0.08, 3),
              "chunglu3k": lambda: synth.chung_lu(3000, 12.0, 2.4, 5, plant_size=25,
                                                  plant_prob=0.85)[:3],
              "rmat2k": lambda: synth.rmat(2048, 16, 9, plant_size=20, plant_prob=1.0)[:3]}
    n, s, d = graphs[name]()
    k, T = 4, 20
    want = O.solve(n, s, d, k, T)
    sct = K.kdss_build_sct(n, s, d, k)
    st = K.kdss_fw_iterate(sct, None, T, K.make_opts(flags=K.KDSS_FLAG_ROOTED))
    r, _ = K.kdss_state_copy_r(st, n, K.KDSS_INT64)
    assert np.array_equal(r, want["r"])
    res = K.kdss_extract(sct, st)
    assert (res["istar"], res["count"]) == (want["istar"], want["count"])
