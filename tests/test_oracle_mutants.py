"""Planted mistakes: each plausible slip in the oracle (a dropped term, a
wrong sign, weight or index, in-place updates) is compiled into a copy of
the oracle on the CPU, and at least one pin must then fail.  This is what
shows the pins are tight enough to trust the oracle."""
import os
import shutil
import subprocess

import pytest

import oracle
from tests import test_oracle_counter as tc
from tests import test_oracle_hyperball as th
from tests import test_oracle_packed as tp
from tests import test_oracle_weights_discount as tw

SRC = os.path.join(os.path.dirname(oracle.__file__), "hb_oracle.c")

MUTANTS = {
    "index_from_low_bits": ("*index = (uint32_t)(x >> (64 - b));",
                            "*index = (uint32_t)(x & ((1ULL << b) - 1));"),
    "rho_without_plus_one": ("uint32_t r = zeros + 1;", "uint32_t r = zeros;"),
    "alpha64": ("if (p == 64) return 0.709;", "if (p == 64) return 0.7213;"),
    "empty_registers_dropped": ("return (double)V + ldexp((double)S, b - 64);",
                                "return ldexp((double)S, b - 64);"),
    "small_range_threshold": ("if (E <= 2.5 * (double)p && V > 0)",
                              "if (E <= 5.0 * (double)p && V > 0)"),
    "small_range_inverted": ("E = (double)p * log((double)p / (double)V);",
                             "E = (double)p * log((double)V / (double)p);"),
    "distance_weight_t": ("sumd[v] = sumd[v] + dist * delta;",
                          "sumd[v] = sumd[v] + (dist - 1.0) * delta;"),
    "harmonic_times_distance": ("harm[v] = harm[v] + delta / dist;",
                                "harm[v] = harm[v] + delta * dist;"),
    "delta_sign": ("double delta = orc_size(a, b) - orc_size(cur + v * p, b);",
                   "double delta = orc_size(cur + v * p, b) - orc_size(a, b);"),
    "in_place_updates": ("memcpy(next + v * p, a, (size_t)p);                  /* write <v, a> */",
                         "memcpy(next + v * p, a, (size_t)p); memcpy((uint8_t *)cur + v * p, a, (size_t)p);"),
    "stop_one_early": ("if (k == 0) { converged = 1; break; }",
                       "if (k <= 1) { converged = 1; break; }"),
    "lin_not_squared": ("if (lin) lin[v] = s > 0.0 ? r * r / s : 1.0;",
                        "if (lin) lin[v] = s > 0.0 ? r / s : 1.0;"),
    "closeness_empty_is_one": ("if (closeness) closeness[v] = s > 0.0 ? 1.0 / s : 0.0;",
                               "if (closeness) closeness[v] = s > 0.0 ? 1.0 / s : 1.0;"),
    "must_check_own_flag": ("if (changed[targets[e]]) { m = 1; break; }",
                            "if (changed[v]) { m = 1; break; }"),
    "replicas_overlap_across_nodes": ("orc_add(c + v * p, b, orc_hash(seed, first + (uint64_t)k));",
                                      "orc_add(c + v * p, b, orc_hash(seed, (uint64_t)v + (uint64_t)k));"),
    "replica_dropped": ("for (int64_t k = 0; k < w[v]; ++k)", "for (int64_t k = 1; k < w[v]; ++k)"),
    "discount_at_distance_t": ("double fdist = disc ? orc_discount(ftable, flen, (int64_t)t + 1) : 0.0;",
                               "double fdist = disc ? orc_discount(ftable, flen, (int64_t)t) : 0.0;"),
    "discount_table_shifted": ("return (d >= 1 && d <= len) ? table[d - 1] : 0.0;",
                               "return (d >= 0 && d < len) ? table[d] : 0.0;"),
    "discount_not_accumulated": ("if (disc) disc[v] = disc[v] + fdist * delta;",
                                 "if (disc) disc[v] = fdist * delta;"),
    "exact_reach_excludes_source": ("reach[k] = (double)tail;", "reach[k] = (double)(tail - 1);"),
    "exact_harmonic_counts_source": ("if (du > 0) { s += (double)du; h += 1.0 / (double)du; }",
                                     "if (du > 0) { s += (double)du; } h += 1.0 / (double)(du + 1);"),
    "exact_ecc_off_by_one": ("if (du > e_max) e_max = du;", "if (du + 1 > e_max) e_max = du + 1;"),
    "packed_high_bit_dropped": ("        for (int bit = 0; bit < 6; ++bit)\n            if ((M[j] >> bit) & 1) {",
                                "        for (int bit = 0; bit < 5; ++bit)\n            if ((M[j] >> bit) & 1) {"),
    "packed_unpack_stride": ("int i = 6 * j + bit;\n            v |=", "int i = 5 * j + bit;\n            v |="),
    "packed_step_reads_unpacked_own": ("orc_unpack6(cur + v * row, b, own);",
                                       "memcpy(own, cur + v * row, (size_t)row); memset(own + row, 0, (size_t)(p - row));"),
    "neighbourhood_skips_a_node": ("for (int64_t v = 0; v < n; ++v) N = N + orc_size(c + v * p, b);",
                                   "for (int64_t v = 1; v < n; ++v) N = N + orc_size(c + v * p, b);"),
}


def _checks(orc):
    """The pins each mutant is run against; a mutant passes only if all pass."""
    yield lambda: tc.test_rho_plus_paper_example(orc)
    for b in (4, 7, 12):
        yield lambda b=b: tc.test_split_crafted_words(orc, b)
        yield lambda b=b: tc.test_size_closed_forms(orc, b)
    yield lambda: tc.test_alpha_constants(orc)
    yield lambda: tc.test_small_range_switch(orc)
    yield lambda: tc.test_register_sum_exact(orc)
    for name in ("path", "zipf", "loops_dups"):
        yield lambda name=name: th.test_counters_equal_hll_of_balls(orc, name, 4, 42)
    yield lambda: th.test_accumulators_closed_form(orc, 40, 12, 2)
    yield lambda: th.test_finalize_special_cases(orc)
    for name in ("zipf", "path"):
        yield lambda name=name: th.test_run_matches_stepwise(orc, name)
    yield lambda: th.test_must_check_definition(orc)
    yield lambda: tw.test_weighted_counters_equal_hll_of_replica_balls(orc, "dag", 4, 42)
    yield lambda: tw.test_weighted_discounted_accumulators_closed_form(orc, "log", 10, 8, 1)
    yield lambda: tw.test_discounts_that_reduce_to_the_accumulators(orc, "dag")
    yield lambda: tw.test_neighbourhood_function_closed_form(orc)
    for name in ("dag", "star_in"):
        yield lambda name=name: th.test_exact_centralities_equal_brute_force_bfs(orc, name, True)
    yield lambda: tp.test_round_trip_every_position_and_value(orc, 6)
    yield lambda: tp.test_packed_counters_equal_hll_of_balls(orc, "path", 4, 42)


def test_unmutated_oracle_passes_every_check(orc):
    for check in _checks(orc):
        check()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(orc, tmp_path, monkeypatch, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", str(path), "-o", str(so), "-lm"], check=True)
    monkeypatch.setattr(oracle, "_lib", oracle._load(str(so)))
    oracle.set_threads(1)
    failed = 0
    for check in _checks(oracle):
        try:
            check()
        except (AssertionError, ValueError):   # a pin fails, or the oracle refuses its own output
            failed += 1
            break
    oracle.set_threads(0)
    assert failed, f"mutant {name} passed every pin"
