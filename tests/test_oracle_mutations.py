"""Plant plausible mistakes in copies of the oracle (on the CPU) and check
that at least one pin fails for each: the pins are strong enough to catch a
dropped term, a wrong sign or index, or a swapped order."""
import os
import subprocess
import sys
import textwrap

import pytest

import oracle

# (name, text in orbg_oracle.c, replacement)
MUTATIONS = [
    ("tie_break_reversed", "(rj == rk && pi[j] > key)", "(rj == rk && pi[j] < key)"),
    ("sort_descending", "if (rj > rk ||", "if (rj < rk ||"),
    ("hard_decision_ge", "llr[i] > 0.0f ? 1 : 0", "llr[i] >= 0.0f ? 1 : 0"),
    ("no_start_syndrome", "d.s0[j] ^= col[(size_t)i * words + j];", "(void)0;"),
    ("zero_pattern_skipped", "rc = fn(NULL, 0, ctx);               /* R = 0",
     "rc = 0;               /* R = 0"),
    ("segments_weight_zero_skipped", "for (R = 0; R <= Rmax && !rc; R++) {",
     "for (R = 1; R <= Rmax && !rc; R++) {"),
    ("build_mountain_step5_dropped", "u[w - q] += r;", "(void)r;"),
    ("landslide_smallest_k", "for (k = w; k >= 1; k--)", "for (k = 1; k <= w; k++)"),
    ("cap_off_by_one", "if (d->t >= d->cap)", "if (d->t > d->cap)"),
    ("hamming_weight_descending", "for (w = 1; w <= n; w++) {", "for (w = n; w >= 1; w--) {"),
    ("rw_divisibility_dropped", "if ((R - J0 * w) % beta)", "if (0)"),
    ("rw_hamming_term_dropped", "L = (R - J0 * w) / beta;", "L = R / beta;"),
    ("rw_slope_on_hamming", "L = (R - J0 * w) / beta;", "L = (R - beta * w) / beta;"),
    ("segment_shift_dropped", "c->v[c->nv++] = base + k + u[k];",
     "c->v[c->nv++] = k + u[k];"),
    ("segment_upper_bound_off", "L <= (long)(ni + 1) * w - (long)w * (w + 1) / 2;",
     "L <= (long)(ni + 2) * w - (long)w * (w + 1) / 2;"),
    ("segment_intercept_ignored", "rem = Wi - (long)w * md->J[i];", "rem = Wi;"),
    ("vu_map_transposed", "v[i] = i + u[i];", "v[i] = i + u[w + 1 - i];"),
    ("flip_wrong_index", "c_out[pi[d.hit_v[i] - 1]] ^= 1;", "c_out[d.hit_v[i] - 1] ^= 1;"),
    ("fit_gap_tie_to_larger_index", "if (g > gap) {", "if (g >= gap && g > 0.0) {"),
    ("fit_split_last_interval", "const int lo = a[0], hi = a[1];",
     "const int lo = a[na - 2], hi = a[na - 1];"),
    ("fit_centre_rounded_up", "a[1] = n / 2;", "a[1] = (n + 1) / 2;"),
    ("fit_Q_largest_slope", "if (s[i] < Q)", "if (s[i] > Q)"),
    ("fit_range_guard_dropped",
     "if (!(s[i] / Q <= ORC_FIT_MAX) || !(L[a[i]] / Q <= ORC_FIT_MAX))", "if (0)"),
    ("fit_first_slope_from_origin", "s[0] = (L[a[1]] - L[1]) / (double)(a[1] - 1);",
     "s[0] = L[a[1]] / (double)a[1];"),
    ("fit_J0_unshifted", "J[0] = orc_round(L[1] / Q) - beta[0];", "J[0] = orc_round(L[1] / Q);"),
    ("fit_J_at_segment_start", "J[i] = orc_round(L[a[i]] / Q);",
     "J[i] = orc_round(L[a[i] + 1] / Q);"),
    ("fit_divisible_floor", "J[i] = orc_round((double)J[i] / (double)beta[i]) * beta[i];",
     "J[i] = (long)floor((double)J[i] / (double)beta[i]) * beta[i];"),
    ("fit_divisible_next_slope", "J[i] = orc_round((double)J[i] / (double)beta[i]) * beta[i];",
     "J[i] = orc_round((double)J[i] / (double)beta[i < m - 1 ? i + 1 : i]) *"
     " beta[i < m - 1 ? i + 1 : i];"),
]

RUNNER = textwrap.dedent("""
    import sys
    sys.path[:0] = [{root!r}, {tests!r}]
    import oracle, oracle_pins
    orc = oracle.Oracle({lib!r})
    failed = []
    for p in oracle_pins.FAST_PINS:
        try:
            p(orc)
        except AssertionError:
            failed.append(p.__name__)
    print("FAILED_PINS", failed)
    sys.exit(1 if failed else 0)
""")


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(tmp_path, name, old, new):
    src = open(oracle.ORACLE_SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / ("orbg_oracle_%s.c" % name)
    mutated.write_text(src.replace(old, new))
    lib = str(tmp_path / ("lib_%s.so" % name))
    oracle.compile_oracle(str(mutated), lib)
    tests_dir = os.path.dirname(os.path.abspath(__file__))
    code = RUNNER.format(root=os.path.dirname(tests_dir), tests=tests_dir, lib=lib)
    # a subprocess: a mutant may misbehave; it must not take pytest with it
    try:
        p = subprocess.run([sys.executable, "-c", code], capture_output=True,
                           text=True, timeout=120)
    except subprocess.TimeoutExpired:
        return  # a mutant that never finishes is caught too
    assert p.returncode != 0, "mutation %s passed every pin:\n%s" % (name, p.stdout)
