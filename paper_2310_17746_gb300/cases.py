"""Run one sieve call from the command line (for timing and profiler captures).

  python -m paper_2310_17746_gb300.cases count  LO HI [--seg W] [--reps R]
  python -m paper_2310_17746_gb300.cases list   LO HI [--reps R]
  python -m paper_2310_17746_gb300.cases primes32 N [--reps R]

Numbers accept Python expressions such as 10**10+1 or 2**30.  Options may
set tile_bits / block_threads / group_hits.  Prints one line per repetition
with the CUDA-event time of the call.
"""
from __future__ import annotations

import argparse
import sys


def _num(s: str) -> int:
    return int(eval(s, {"__builtins__": {}}, {}))  # literal arithmetic only


def main(argv=None) -> int:
    import torch

    from . import binding

    ap = argparse.ArgumentParser()
    ap.add_argument("kind", choices=["count", "list", "primes32"])
    ap.add_argument("a", type=_num)
    ap.add_argument("b", type=_num, nargs="?")
    ap.add_argument("--seg", type=_num, default=0)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--tile-bits", type=_num, default=0)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--group-hits", type=int, default=0)
    args = ap.parse_args(argv)

    hi = args.b if args.kind in ("count", "list") else args.a + 1
    lo = args.a if args.kind in ("count", "list") else 0
    sv = binding.Sieve(max(hi, 2))
    opts = {k: v for k, v in (("tile_bits", args.tile_bits), ("block_threads", args.block_threads),
                              ("group_hits", args.group_hits)) if v}
    if opts:
        sv.set_options(**opts)
    dev = torch.device("cuda")
    st = torch.cuda.current_stream()
    if args.kind == "count":
        if args.seg:
            nb = binding.Sieve.nbins(lo, hi, args.seg)
            counts = torch.zeros(max(nb, 1), dtype=torch.int64, device=dev)
        total = torch.zeros(2, dtype=torch.int64, device=dev)
    elif args.kind == "list":
        cap = sv.range_count(lo, hi).count
        out = torch.zeros(max(cap, 1), dtype=torch.int64, device=dev)
    else:
        cap = sv.count(args.a).count
        out = torch.zeros(max(cap, 1), dtype=torch.int32, device=dev)
    for r in range(args.reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(st)
        if args.kind == "count":
            if args.seg:
                sv.segment_counts(lo, hi, args.seg, counts=counts[:nb], total=total)
            else:
                sv.range_count(lo, hi, out=total)
            res = int(total[0])
        elif args.kind == "list":
            res = sv.range_list(lo, hi, out=out)
        else:
            res = sv.primes(args.a, out=out)
        e.record(st)
        torch.cuda.synchronize()
        print(f"{args.kind} [{lo}, {hi}) rep {r}: {res} primes, {s.elapsed_time(e):.3f} ms", flush=True)
    sv.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
