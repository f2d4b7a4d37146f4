"""Run one sieve call from the command line (for timing and profiler captures).

  python -m paper_2310_17746_gb300.cases count  LO HI [--seg W] [--reps R]
  python -m paper_2310_17746_gb300.cases list   LO HI [--reps R]
  python -m paper_2310_17746_gb300.cases primes32 N [--reps R]
  python -m paper_2310_17746_gb300.cases batch  NQ [--seed S] [--count-only] [--mix batch|serving] [--reps R]

Numbers accept Python expressions such as 10**10+1 or 2**30.  Options may
set tile_bits / block_threads / group_hits / presieve_groups, the bucket
sieve's threshold, wave and scatter kind, and the one-pass list.  Prints one
line per repetition with the CUDA-event time of the call.
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
    ap.add_argument("kind", choices=["count", "list", "primes32", "batch"])
    ap.add_argument("a", type=_num)
    ap.add_argument("b", type=_num, nargs="?")
    ap.add_argument("--seg", type=_num, default=0)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--tile-bits", type=_num, default=0)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--group-hits", type=int, default=0)
    ap.add_argument("--presieve-groups", type=int, default=-1)
    ap.add_argument("--bucket-threshold", type=int, default=-1, help="0 turns the bucket sieve off")
    ap.add_argument("--bucket-wave", type=int, default=0)
    ap.add_argument("--bucket-scatter", type=int, default=-1, help="0 automatic, 1 direct, 2 sorted")
    ap.add_argument("--single-pass", type=int, default=-1, help="list: 1 one pass, 0 two passes")
    ap.add_argument("--cluster-ctas", type=int, default=-1, help="0 off, 2/4/8/16: cluster segments")
    ap.add_argument("--cluster-threshold", type=int, default=-1)
    ap.add_argument("--batch-tile-bits", type=_num, default=0)
    ap.add_argument("--chunk-primes", type=_num, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--count-only", action="store_true")
    ap.add_argument("--naive", action="store_true", help="batch: one range launch per query")
    ap.add_argument("--mix", choices=["batch", "serving"], default="batch",
                    help="batch: the 4096-query batch workload's distribution; serving: the serving "
                         "workload's (lo up to 1e18, width up to 1e9, seed 1)")
    args = ap.parse_args(argv)
    if args.kind == "batch":
        return _batch(args)

    hi = args.b if args.kind in ("count", "list") else args.a + 1
    lo = args.a if args.kind in ("count", "list") else 0
    sv = binding.Sieve(max(hi, 2))
    opts = {k: v for k, v in (("tile_bits", args.tile_bits), ("block_threads", args.block_threads),
                              ("group_hits", args.group_hits), ("bucket_wave", args.bucket_wave)) if v}
    opts.update({k: v for k, v in (("presieve_groups", args.presieve_groups),
                                   ("bucket_threshold", args.bucket_threshold),
                                   ("bucket_scatter", args.bucket_scatter),
                                   ("list_single_pass", args.single_pass),
                                   ("cluster_ctas", args.cluster_ctas),
                                   ("cluster_threshold", args.cluster_threshold)) if v >= 0})
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


def _batch(args) -> int:
    """The batched-range workload (log-uniform lo in [1e6, 1e15], width in
    [1e3, 1e8], half list mode), or the serving mix's queries (lo in [1e6,
    1e18], width in [1e3, 1e9], list with probability 0.2), with device
    outputs."""
    import numpy as np
    import torch

    from . import binding, workloads

    if args.mix == "serving":
        q = workloads.serving_arrivals(1000.0, args.a, seed=args.seed or 1).queries
    else:
        q = workloads.batch_queries(n=args.a, seed=args.seed)
    if args.count_only:
        q.mode[:] = workloads.MODE_COUNT
    nq = len(q)
    sv = binding.Sieve(int(q.hi.max()) + 1)
    opts = {k: v for k, v in (("batch_tile_bits", args.batch_tile_bits), ("block_threads", args.block_threads),
                              ("chunk_primes", args.chunk_primes), ("group_hits", args.group_hits)) if v}
    if args.presieve_groups >= 0:
        opts["presieve_groups"] = args.presieve_groups
    if opts:
        sv.set_options(**opts)
    cnt = torch.zeros((nq, 2), dtype=torch.int64, device="cuda")
    off = torch.zeros(nq + 1, dtype=torch.int64, device="cuda")
    cnt_h, _, _ = sv.range_batch(q.lo, q.hi, np.zeros(nq, np.uint8))
    need = int(cnt_h[q.mode == workloads.MODE_LIST, 0].astype(np.int64).sum())
    vals = torch.empty(max(need, 1), dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    for r in range(args.reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(st)
        n = sv.range_batch(q.lo, q.hi, q.mode, cnt=cnt, offsets=off, values=vals, naive=args.naive)
        e.record(st)
        torch.cuda.synchronize()
        print(f"batch {nq} queries rep {r}: {n} listed, {s.elapsed_time(e):.3f} ms", flush=True)
    sv.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
