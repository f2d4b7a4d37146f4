#!/usr/bin/env python
"""Writes tests/golden/count_1e12_bins.json with the CPU oracle only.

The file holds the expected result of the headline workload -- the primes of
[2, 1e12] counted per 2^30-number block (932 blocks; block s is the value
interval [s 2^30, (s+1) 2^30), reading A8) -- together with the count and
the sum of those primes mod 2^64.  Every number in it comes from
oracle.segment_counts (the plain byte sieve of Section 1.1 / Figure 1 on a
range); nothing comes from the CUDA path.  Before writing, the script checks
the oracle's totals against the published values: pi(10^12) = 37607912018
(OEIS A006880) and the sum of the primes below 10^12,
18435588552550705911377 (OEIS A046731), reduced mod 2^64.

  python tests/golden/make_count_1e12_bins.py      # a few minutes on 8-16 cores
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LO, HI, SEG = 2, 10**12 + 1, 1 << 30
PI_1E12 = 37607912018                       # OEIS A006880
SUM_BELOW_1E12 = 18435588552550705911377    # OEIS A046731


def main() -> int:
    import oracle

    t = time.perf_counter()
    base = oracle.base_table(10**6)
    count, checksum, bins = oracle.segment_counts(LO, HI, SEG, base=base)
    dt = time.perf_counter() - t
    if count != PI_1E12 or checksum != SUM_BELOW_1E12 % 2**64 or int(bins.sum()) != count:
        print(f"oracle disagrees with the published values: {count} {checksum}", file=sys.stderr)
        return 1
    doc = {
        "citation": "Expected result of the headline count: primes of [2, 1e12] per 2^30-number block "
                    "(block s = values [s*2^30, (s+1)*2^30), reading A8). Bins and checksum written by "
                    "tests/golden/make_count_1e12_bins.py from the CPU oracle only (oracle.segment_counts); "
                    "the totals agree with OEIS A006880 (pi(10^12)) and OEIS A046731 (sum of the primes "
                    "below 10^12 = 18435588552550705911377, here mod 2^64).",
        "lo": LO, "hi_exclusive": HI, "seg_width": SEG,
        "count": count, "checksum_mod_2_64": checksum, "sum_below_1e12": SUM_BELOW_1E12,
        "bins": [int(x) for x in bins],
        "oracle_seconds": round(dt, 1), "oracle_threads": oracle.default_threads(),
    }
    with open(os.path.join(HERE, "count_1e12_bins.json"), "w") as f:
        json.dump(doc, f, indent=0)
        f.write("\n")
    print(f"wrote {len(bins)} bins, count {count}, checksum {checksum} in {dt:.0f} s")
    return 0


if __name__ == "__main__":
    sys.exit(main())
