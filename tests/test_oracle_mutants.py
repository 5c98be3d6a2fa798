"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake in a temporary copy of the oracle's C source (a
dropped term, a wrong index, a flipped tie-break, an off-by-one), builds it,
swaps it in, and checks that at least one pin of test_oracle_pins fails.  The
committed oracle is never modified.

The pivot tie-break of the SCT recursion is not among the cases: any pivot
yields a valid SCT and the paper's example is tie-free, so no fact of the
paper fixes it; it is a convention that the CUDA parity tests cover.
"""
import ctypes
import os
import subprocess

import pytest

import oracle as O
import test_oracle_pins as P

try:   # the CPSample pins compare with networkx
    import test_oracle_cpsample as CP
except ImportError:  # pragma: no cover - networkx missing
    CP = None

MUTANTS = {
    "pivot_cap_drops_the_minus_one": (
        "uint64_t up_p = orc_binom(p - 1, k - h - 1, &ovf);",
        "uint64_t up_p = orc_binom(p, k - h - 1, &ovf);"),
    "zero_cap_nodes_kept_in_plateaus": (
        "if (up[i] > 0) srt[ns++] = i;\n    g_sort_r = r_in;",
        "srt[ns++] = i;\n    g_sort_r = r_in;"),
    "remainder_to_highest_id": (
        "for (uint64_t j = 0; j < nC; ++j) { r[A[j]] += 1; up[A[j]] -= 1; }",
        "for (uint64_t j = 0; j < nC; ++j) { r[A[na - 1 - j]] += 1; up[A[na - 1 - j]] -= 1; }"),
    "hold_branch_keeps_handled_candidates": (
        "for (int j = 0; j < ncur; ++j) if (cur[j] != w) cur[q++] = cur[j];",
        "for (int j = 0; j < ncur; ++j) cur[q++] = cur[j];"),
    "prefix_event_one_position_early": (
        "acc[mh + 1] += prev;", "acc[mh] += prev;"),
    "alg1_sync_ties_to_highest_id": (
        "if (r[u] < r[best] || (r[u] == r[best] && u < best)) best = u;",
        "if (r[u] < r[best] || (r[u] == r[best] && u > best)) best = u;"),
    "argmax_ties_to_smallest_prefix": (
        "if (frac_cmp(a, (uint64_t)i, b, (uint64_t)best) >= 0) best = i;",
        "if (frac_cmp(a, (uint64_t)i, b, (uint64_t)best) > 0) best = i;"),
    "clique_listing_skips_a_candidate": (
        "for (int64_t j = i + 1; j < nc; ++j)\n            if (is_adj(c->off, c->adj, v, cand[j]))",
        "for (int64_t j = i + 2; j < nc; ++j)\n            if (is_adj(c->off, c->adj, v, cand[j]))"),
    "binomial_off_by_one": (
        "u128 f = (u128)(a - b + i), x = v, y = (u128)i;",
        "u128 f = (u128)(a - b + i + 1), x = v, y = (u128)i;"),
    "cont_delta_not_cleared_between_iterations": (
        "++t) {\n        memset(dr, 0, sizeof(double) * (size_t)n);", "++t) {\n"),
    "cont_pairs_update_r_in_place": (
        "rc = orc_pbupdate_cont(len, ids, rv, hcnt[q], k, dv);\n            if (rc) break;\n"
        "            for (int i = 0; i < len; ++i) dr[ids[i]] += dv[i];",
        "rc = orc_pbupdate_cont(len, ids, rv, hcnt[q], k, dv);\n            if (rc) break;\n"
        "            for (int i = 0; i < len; ++i) r[ids[i]] += dv[i];"),
    "seq_reads_the_previous_iterate": (
        "            for (int i = 0; i < len; ++i) rv[i] = r[ids[i]];\n"
        "            rc = orc_pbupdate_alg3(len, ids, rv, hcnt[q], k, dv);\n"
        "            if (rc) break;\n"
        "            for (int i = 0; i < len; ++i) r[ids[i]] += dv[i];",
        "            if (q == 0) { static uint64_t *snap; snap = (uint64_t *)realloc(snap, "
        "sizeof(uint64_t) * (size_t)(n + 1)); memcpy(snap, r, sizeof(uint64_t) * (size_t)n); "
        "g_snap = snap; }\n"
        "            for (int i = 0; i < len; ++i) rv[i] = g_snap[ids[i]];\n"
        "            rc = orc_pbupdate_alg3(len, ids, rv, hcnt[q], k, dv);\n"
        "            if (rc) break;\n"
        "            for (int i = 0; i < len; ++i) r[ids[i]] += dv[i];"),
    "rho_prime_pair_enters_before_its_pivot_nodes": (
        "int32_t mall = mh;\n        for (int j = 0; j < p; ++j) if (pp[j] > mall) mall = pp[j];",
        "int32_t mall = mh;"),
    "rho_prime_counts_one_per_pair": (
        "facc[mall + 1] += binom128(p, k - h);", "facc[mall + 1] += 1;"),
    # the round counter moves only when the level rises, so the rounds of one
    # level merge (cores stay right; the order of the SCT build changes)
    "peel_round_advances_only_with_the_level": (
        "            c = mn;\n"
        "            continue;\n"
        "        }\n"
        "        for (int64_t i = 0; i < ns; ++i) {\n"
        "            alive[S[i]] = 0; core[S[i]] = (int32_t)c; round_out[S[i]] = (int32_t)rnd;\n"
        "        }\n"
        "        for (int64_t i = 0; i < ns; ++i) {\n"
        "            int32_t v = S[i];\n"
        "            for (int64_t e = off[v]; e < off[v + 1]; ++e)\n"
        "                if (alive[adj[e]]) deg[adj[e]]--;\n"
        "        }\n"
        "        if (c > maxcore) maxcore = c;\n"
        "        removed += ns;\n"
        "        rnd++;\n",
        "            c = mn;\n"
        "            rnd++;\n"
        "            continue;\n"
        "        }\n"
        "        for (int64_t i = 0; i < ns; ++i) {\n"
        "            alive[S[i]] = 0; core[S[i]] = (int32_t)c; round_out[S[i]] = (int32_t)rnd;\n"
        "        }\n"
        "        for (int64_t i = 0; i < ns; ++i) {\n"
        "            int32_t v = S[i];\n"
        "            for (int64_t e = off[v]; e < off[v + 1]; ++e)\n"
        "                if (alive[adj[e]]) deg[adj[e]]--;\n"
        "        }\n"
        "        if (c > maxcore) maxcore = c;\n"
        "        removed += ns;\n"),
    "final_sort_u64_ties_to_descending_ids": (
        "if (g_key_u[x] != g_key_u[y]) return g_key_u[x] > g_key_u[y] ? -1 : 1;\n    return x < y ? -1 : x > y;",
        "if (g_key_u[x] != g_key_u[y]) return g_key_u[x] > g_key_u[y] ? -1 : 1;\n    return x > y ? -1 : x < y;"),
    "final_sort_f64_ties_to_descending_ids": (
        "if (g_key_d[x] != g_key_d[y]) return g_key_d[x] > g_key_d[y] ? -1 : 1;\n    return x < y ? -1 : x > y;",
        "if (g_key_d[x] != g_key_d[y]) return g_key_d[x] > g_key_d[y] ? -1 : 1;\n    return x > y ? -1 : x < y;"),
    # the synchronous iterations add each pair's units into r at once, so later
    # pairs of the iteration read them (the in-place form of Alg. 2)
    "sync_pairs_update_r_in_place": (
        "            for (int i = 0; i < len; ++i) dr[ids[i]] += dv[i];\n"
        "        }\n"
        "        for (int64_t v = 0; v < n; ++v) r[v] += dr[v];\n"
        "    }\n"
        "    free(dr); free(rv); free(dv);\n"
        "    return rc;\n"
        "}\n"
        "\n"
        "/* The synchronous iterations of orc_fw_sync with",
        "            for (int i = 0; i < len; ++i) r[ids[i]] += dv[i];\n"
        "        }\n"
        "        for (int64_t v = 0; v < n; ++v) r[v] += 0;\n"
        "    }\n"
        "    free(dr); free(rv); free(dv);\n"
        "    return rc;\n"
        "}\n"
        "\n"
        "/* The synchronous iterations of orc_fw_sync with"),
    # the synchronous iterations keep summing into the previous iteration's delta
    "sync_delta_not_cleared": (
        "    for (int t = 1; t <= T && rc == ORC_OK; ++t) {\n"
        "        memset(dr, 0, sizeof(uint64_t) * (size_t)n);\n"
        "        for (int64_t q = 0; q < npairs; ++q) {\n"
        "            int len = (int)(pair_off[q + 1] - pair_off[q]);\n"
        "            const int32_t *ids = nodes + pair_off[q];\n"
        "            for (int i = 0; i < len; ++i) rv[i] = r[ids[i]];\n"
        "            rc = orc_pbupdate_alg3(",
        "    memset(dr, 0, sizeof(uint64_t) * (size_t)n);\n"
        "    for (int t = 1; t <= T && rc == ORC_OK; ++t) {\n"
        "        for (int64_t q = 0; q < npairs; ++q) {\n"
        "            int len = (int)(pair_off[q + 1] - pair_off[q]);\n"
        "            const int32_t *ids = nodes + pair_off[q];\n"
        "            for (int i = 0; i < len; ++i) rv[i] = r[ids[i]];\n"
        "            rc = orc_pbupdate_alg3("),
    # CPSample (Alg. 4): colours taken in ascending instead of descending
    # rank; the sample rank drawn from 52 instead of 53 bits of the word
    "colour_in_rank_ascending": (
        "qsort(ord, (size_t)n, sizeof(int32_t), cmp_rank_desc);",
        "qsort(ord, (size_t)n, sizeof(int32_t), cmp_key);"),
    "sample_rank_uses_52_bits": (
        "uint64_t R = (uint64_t)(((unsigned __int128)(x >> 11) * tot) >> 53);",
        "uint64_t R = (uint64_t)(((unsigned __int128)(x >> 12) * tot) >> 53);"),
    "plateau_gap_ignored": (
        "if (gap < w) w = gap;\n            if (nC / (uint64_t)na < w)",
        "if (nC / (uint64_t)na < w)"),
}

PINS = [
    P.test_g1_triangles_and_densest_subgraph,
    P.test_g1_sct_matches_example_2_2,
    P.test_g1_example_3_1_pbupdate_steps,
    P.test_g1_psctl_extracts_densest,
    P.test_g1_converges_to_sct_cp_optimum,
    lambda: P.test_sct_partitions_the_k_cliques(O.ORDER_PEEL),
    P.test_pbupdate_is_an_optimal_integer_allocation,
    P.test_fw_invariants_and_weak_duality,
    P.test_prefix_counts_from_pairs_equal_explicit_list,
    P.test_argmax_takes_the_largest_prefix_on_ties,
    lambda: P.test_brute_force_small_graphs(3),
    P.test_alg1_synchronous_over_explicit_cliques,
    P.test_g1_inplace_iterations_match_hand_trace,
    P.test_g1_continuous_iterations_match_hand_trace,
    P.test_g1_continuous_rule_converges_to_sct_cp_optimum,
    P.test_fw_cont_and_fw_seq_invariants_and_weak_duality,
    P.test_rho_prime_prefix_counts_equal_their_definition,
    P.test_peel_rounds_satisfy_their_definition,
    P.test_final_sort_is_r_descending_with_ties_to_ascending_ids,
]
CPSAMPLE_MUTANTS = {"colour_in_rank_ascending", "sample_rank_uses_52_bits"}
if CP is not None:
    PINS += [lambda: CP.test_greedy_colouring_is_networkx_greedy_in_the_same_order(1),
             lambda: CP.test_each_sample_is_the_path_of_its_rank(1),
             CP.test_cpsample_finds_the_example_densest_subgraph]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path, monkeypatch):
    if name in CPSAMPLE_MUTANTS and CP is None:
        pytest.skip("the CPSample pins need networkx")
    old, new = MUTANTS[name]
    src = open(O.SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / "mutant.c"
    mutated = src.replace(old, new)
    if "g_snap" in new:   # the stale-read mutant keeps its snapshot pointer at file scope
        mutated = mutated.replace("int orc_fw_seq(", "static const uint64_t *g_snap;\nint orc_fw_seq(", 1)
    path.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", str(so),
                           str(path), "-lm"])
    real = O.lib()
    mutant = ctypes.CDLL(str(so))
    # copy the ctypes signatures of the real library onto the mutant
    for attr in dir(real):
        if attr.startswith("orc_"):
            f, g = getattr(real, attr), getattr(mutant, attr)
            g.argtypes, g.restype = f.argtypes, f.restype
    monkeypatch.setattr(O, "_lib", mutant)
    caught = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, OverflowError, ValueError):
            caught.append(getattr(pin, "__name__", "pin"))
    assert caught, f"no pin failed for planted mistake {name}"
