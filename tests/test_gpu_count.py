"""The count-only SCT pass (kdss_sct_count): the sizes of P_k without storing
a pair (Sec. 2, Lemmas 2.4-2.6; Thm 3.7's O(eta) space is what it measures).

- Unbudgeted, it equals the sizes of the k-pruned build exactly.
- On the complete graph K_1100 (k = 8) every root's recursion is one pivot
  chain, so P_k is known in closed form: root i (in id order, the peel order
  of a regular graph) holds ({i}, its 1099 - i later vertices), kept while
  1100 - i >= k, and c_k = C(1100, 8) by the hockey-stick identity -- above
  2^64, with 76 pairs longer than the FW kernels' 1024 nodes (the k-pruned
  build refuses that graph).
- With a time budget it stops early, counts only the roots it walked to the
  end, and never more than the whole SCT.
"""
import math

import numpy as np
import pytest

import paper_2403_05775_gb300 as K
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    K.load(build_if_missing=True)


GRAPHS = {
    "er300": lambda: synth.erdos_renyi(300, 0.08, 3),
    "chunglu3k": lambda: synth.chung_lu(3000, 12.0, 2.4, 5, plant_size=25, plant_prob=0.85)[:3],
    "rmat2k": lambda: synth.rmat(2048, 16, 9, plant_size=20, plant_prob=1.0)[:3],
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [3, 4, 6])
def test_count_equals_the_build(name, k):
    n, s, d = GRAPHS[name]()
    sct = K.kdss_build_sct(n, s, d, k)
    info = K.kdss_sct_info(sct)
    cnt = K.kdss_sct_count(n, s, d, k)
    assert cnt["complete"] == 1 and cnt["roots_done"] == n and cnt["roots_cut"] == 0
    assert cnt["eta_k"] == info["eta_k"] and cnt["L_k"] == info["L_k"]
    assert cnt["c_k"] == info["c_k"]
    assert cnt["pairs_per_class"][:5] == info["pairs_per_class"][:5]
    assert cnt["pairs_per_class"][5] == 0
    assert cnt["max_pair_len"] == info["max_pair_len"]
    assert cnt["degeneracy"] == info["degeneracy"] and cnt["m"] == info["m"]


def test_count_of_the_complete_graph_closed_form():
    m, k = 1100, 8
    iu = np.triu_indices(m, 1)
    s, d = iu[0].astype(np.int32), iu[1].astype(np.int32)
    cnt = K.kdss_sct_count(m, s, d, k)
    assert cnt["complete"] == 1
    assert cnt["eta_k"] == m - k + 1
    assert cnt["L_k"] == sum(range(k, m + 1))
    assert cnt["c_k"] == math.comb(m, k) and cnt["c_k"] >= 2 ** 64
    assert cnt["pairs_per_class"][5] == m - 1024
    assert cnt["max_pair_len"] == m and cnt["max_out_degree"] == m - 1
    with pytest.raises(K.KdssError) as e:
        K.kdss_build_sct(m, s, d, k)
    assert e.value.code == K.KDSS_ERR_UNSUPPORTED


def test_count_with_a_time_budget_stops_early():
    n, s, d = synth.workload_chunglu_1e5()
    full = K.kdss_sct_count(n, s, d, 5)
    assert full["complete"] == 1
    part = K.kdss_sct_count(n, s, d, 5, budget_s=1e-5)
    assert part["complete"] == 0
    assert part["roots_done"] + part["roots_cut"] <= n
    assert 0 <= part["eta_k"] <= full["eta_k"] and part["L_k"] <= full["L_k"]
    assert part["c_k"] <= full["c_k"]
