"""Planted mistakes in the oracle must be caught by the pins (CPU only).

Each case copies oracle.c, changes one line into a plausible bug (a reversed
tie-break, a wrong sign rule, a signed/unsigned mix-up, an off-by-one), builds
the copy into a temporary library and runs the pin checks of tests/_pins.py
against it: at least one check has to fail.  The real oracle is untouched.
"""
import os

import pytest

import oracle
from oracle import build as obuild
import _pins

MUTATIONS = {
    "tiebreak_reversed": ("return cmp_unsigned(x->idx, y->idx); /* Section 2 tie-break */",
                          "return cmp_unsigned(y->idx, x->idx); /* Section 2 tie-break */"),
    "negatives_ascending": ("return cmp_unsigned(mag_b, mag_a);     /* negatives",
                            "return cmp_unsigned(mag_a, mag_b);     /* negatives"),
    "sign_rule_flipped": ("return neg_a ? -1 : 1;", "return neg_a ? 1 : -1;"),
    "i32_as_unsigned": ("case ORC_I32: return cmp_signed32(a, b);",
                        "case ORC_I32: return cmp_unsigned(a & 0xffffffffu, b & 0xffffffffu);"),
    "bf16_wrong_width": ("cmp_total_order(a & 0xffffu, b & 0xffffu, 16)",
                         "cmp_total_order(a & 0xffffu, b & 0xffffu, 32)"),
    "kth_off_by_one": ("*kth_idx = (uint32_t)v[k - 1].idx;",
                       "*kth_idx = (uint32_t)v[k > 1 ? k - 2 : 0].idx;"),
    "runs_pos_off_by_one": ("*kth_pos = g - run_off[r];", "*kth_pos = g - run_off[r] + 1;"),
    "runs_bisection_strict": ("if (run_off[mid] <= g)", "if (run_off[mid] < g)"),
    "delete_ignores_cursor": ("for (i = run_off[r] + cursor[r]; i < run_off[r + 1]; ++i) {",
                              "for (i = run_off[r]; i < run_off[r + 1]; ++i) {"),
    "freq_tiebreak_reversed": ("return x->obj < y->obj ? -1 : x->obj > y->obj ? 1 : 0;",
                               "return x->obj < y->obj ? 1 : x->obj > y->obj ? -1 : 0;"),
    "ec_counts_sample_only": ("            freq[lo].count += 1;", "            freq[lo].count += mask[i];"),
    "philox_lanes_swapped": ("        c1 = lo1;\n", "        c1 = lo0;\n"),
    "pac_rate_first_term_only": ("rho_n = 4.0 / (eps * eps) * (a > b ? a : b);", "rho_n = 4.0 / (eps * eps) * a;"),
    "largest_ties_reversed": ("        return cmp_unsigned(x->idx, y->idx);                             \\\n",
                              "        return cmp_unsigned(y->idx, x->idx);                             \\\n"),
    "ec_natural_log_of_p": ("ks = sqrt(2.0 * log2((double)pes) / pes * log(n / delta)) / eps;",
                            "ks = sqrt(2.0 * log((double)pes) / pes * log(n / delta)) / eps;"),
    "ec_factor_two_dropped": ("ks = sqrt(2.0 * log2((double)pes) / pes * log(n / delta)) / eps;",
                              "ks = sqrt(log2((double)pes) / pes * log(n / delta)) / eps;"),
    "pac_first_term_2n": ("double a = 3.0 / k * log(4.0 * n / delta);",
                          "double a = 3.0 / k * log(2.0 * n / delta);"),
    "pairs_before_ties_inclusive": ("if (d < 0 || (d == 0 && i < pos))", "if (d < 0 || (d == 0 && i <= pos))"),
    "checker_rank_loose": ("if (before != k - 1)\n        return 1;", "if (before > k)\n        return 1;"),
    "checker_no_bound": ("if (d > 0 || (d == 0 && x > kth)) {", "if (d > 0) {"),
    "take_k_minus_one": ("for (i = 0; i < k; ++i)             /* ranks 1..k */",
                         "for (i = 1; i < k; ++i)             /* ranks 1..k */"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(obuild.SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique in oracle.c"
    mutant_src = tmp_path / "oracle_mutant.c"
    mutant_src.write_text(src.replace(old, new))
    lib = obuild.compile_source(str(mutant_src), str(tmp_path / f"lib_{name}.so"))
    orc = oracle.Oracle(lib)
    failures = []
    for check in _pins.ALL_CHECKS:
        try:
            failures += check(orc)
        except Exception as e:  # a crash on garbage output also counts as caught
            failures.append(f"{check.__name__}: {e!r}")
        if failures:
            break
    assert failures, f"planted mistake {name} passed every pin"
