"""Plant plausible mistakes in a copy of the oracle and show the pins catch each.

Each mutant is oracle.c with one textual change, compiled into a temporary
library.  The test passes when at least one pin check fails on the mutant; a
mutant that survives every check would mean the pins cannot see that mistake.
"""
import os
import shutil

import pytest

import oracle
import oracle_checks as C
from oracle import build as obuild

MUTANTS = {
    # Section 2.4: sieving a prime must start at its square
    "no_square_start": ("      if (m < p * p) m = p * p;\n", ""),
    # base primes needed up to isqrt(hi - 1): stop one too early
    "base_cutoff_off_by_one": ("if (p * p > e - 1) break;", "if (p * p >= e - 1) break;"),
    # primes <= n: the crossing-off primes must reach isqrt(n), not stop one short
    "upto_base_bound_short": ("  const uint64_t r = oracle_isqrt(n);\n", "  const uint64_t r = oracle_isqrt(n) - 1;\n"),
    # keeps 0 and 1 as primes
    "keeps_one": ("if (!seg[i] || v < 2) continue;", "if (!seg[i] || v < 1) continue;"),
    # bins counted from lo instead of from multiples of the width
    "bins_from_lo": ("job->bins[v / job->seg_width - first_bin]++;",
                     "job->bins[(v - job->lo) / job->seg_width]++;"),
    # Miller-Rabin squaring loop one short
    "mr_short_loop": ("for (int j = 1; j < s; j++) {", "for (int j = 2; j < s; j++) {"),
    # isqrt through double-precision sqrt (wrong once n needs more than 53 bits)
    "isqrt_via_double": ("  if (n < 2) return n;\n  int bits", "  if (n < 2) return n;\n  return (uint64_t)__builtin_sqrt((double)n);\n  int bits"),
    # first multiple rounded down instead of up (can start below M)
    "first_multiple_floor": ("uint64_t v = ((M + P - 1) / P) * P;", "uint64_t v = (M / P) * P;"),
}

# checks cheap enough to run on every mutant (the 1e9 / 1e10 runs are skipped)
CHECKS = [C.check_isqrt, C.check_primes_upto_small, C.check_range_small_bruteforce,
          C.check_invariants, C.check_segment_bins, C.check_mr_vs_td,
          C.check_first_class_multiple, C.check_figure2]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(os.path.join(obuild.HERE, "oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    d = tmp_path / "src"
    d.mkdir()
    (d / "oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(obuild.HERE, "oracle.h"), d / "oracle.h")
    lib = obuild.compile_sources(str(d), str(tmp_path / "libmutant.so"))
    m = oracle.Oracle(lib)
    caught = []
    for check in CHECKS:
        try:
            check(m)
        except AssertionError:
            caught.append(check.__name__)
            break
        except oracle.OracleError:
            caught.append(check.__name__ + " (error)")
            break
    assert caught, f"mutant {name} passed every pin"
