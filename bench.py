#!/usr/bin/env python
"""Benchmark of the GB300 segmented sieve.

Headline: sieved range width per second for the count of [2, 1e12] with its
per-2^30-number block histogram (one step = one pass of the whole hot path:
wheel presieve, Table 1 start offsets, strikes, fix-ups, popcount, checksum,
histogram).  Under torchrun each rank sieves its own 1e12-wide range (weak
scaling, no collective on the data path); rank 0 prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle on bounded samples of the same workload
(the only other place this file runs the oracle is the cpu_baseline leg).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sieved range width/s at n=1e12 (count); batched range queries/s; p99 latency"
UNIT = "numbers/s"
WIDTH = 10**12
SEG_WIDTH = 1 << 30
PI_1E12 = 37607912018  # published value (OEIS A006880), checked on every run
TUNE_CACHE = os.path.join(ROOT, "paper_2310_17746_gb300", "tuned_options.json")
TUNE_WORKLOAD = "count 1e12-wide range, 2^30-number blocks"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-queries leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-list", action="store_true", help="skip the list leg")
    ap.add_argument("--no-naive", action="store_true", help="skip the plain GPU sieve comparison")
    ap.add_argument("--no-far", action="store_true", help="skip the far-range (bucket sieve) leg")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def range_cost_ms(lo: int, hi: int) -> float:
    """Modelled count time of [lo, hi) (the library's sharding cost model)."""
    from paper_2310_17746_gb300 import shard
    return shard.cost_ms(lo, hi)


_RANK_RANGES: list[tuple[int, int]] = []


def rank_range(rank: int) -> tuple[int, int]:
    """Rank 0 sieves [2, 1e12] (the headline configuration); rank r > 0 the
    next contiguous range whose modelled count time equals rank 0's, so that
    the work per GPU stays fixed as ranks are added (weak scaling) and the
    ranks finish together.  Widths are multiples of 6e6."""
    if not _RANK_RANGES:
        _RANK_RANGES.append((2, WIDTH + 1))
    while len(_RANK_RANGES) <= rank:
        target = range_cost_ms(*_RANK_RANGES[0])
        lo = _RANK_RANGES[-1][1]
        a, b = 1, WIDTH // 6_000_000  # width in units of 6e6: the cost grows with it
        while a < b:
            m = (a + b + 1) // 2
            if range_cost_ms(lo, lo + m * 6_000_000) <= target:
                a = m
            else:
                b = m - 1
        _RANK_RANGES.append((lo, lo + a * 6_000_000))
    return _RANK_RANGES[rank]


# ---------------------------------------------------------------- accounting

def small_primes(n: int):
    """Primes <= n with a plain numpy sieve (host-side work accounting only)."""
    import numpy as np
    a = np.ones(n + 1, dtype=bool)
    a[:2] = False
    for i in range(2, int(n**0.5) + 1):
        if a[i]:
            a[i * i::i] = False
    return np.nonzero(a)[0].astype(np.int64)


# largest prime removed by the presieve patterns, by presieve_groups
LAST_PRESIEVED = [19, 31, 43, 59, 71, 83, 101, 109, 131]


def algorithmic_ops(lo: int, hi: int, first: int = 23) -> dict:
    """Strikes a segmented 6k+-1 sieve must make on [lo, hi) once the primes
    below `first` are presieved: class-1 and class-5 multiples m of each base
    prime first <= p <= isqrt(hi-1) with max(lo, p^2) <= m < hi; words =
    candidate bits / 32, each written once (presieve) and read once (count)."""
    import numpy as np
    s = math.isqrt(hi - 1)
    p = small_primes(s)
    p = p[p >= first]
    strikes = 0
    a = np.maximum(lo, p * p)
    jmax = (hi - 1) // p
    jmin = (a + p - 1) // p
    for r in (1, 5):
        jr = (r * p) % 6           # class-r multiples p*j have j = r*p (mod 6)
        j0 = jmin + (jr - jmin) % 6
        cnt = np.where(j0 <= jmax, (jmax - j0) // 6 + 1, 0)
        strikes += int(cnt.sum())
    candidates = 2 * ((hi - lo) // 6)
    words = candidates // 32
    return {"strikes": strikes, "candidate_words": words, "ops": strikes + 2 * words}


def source_hash() -> str:
    h = hashlib.sha256()
    # the files the count kernel is compiled from
    for name in ("range.cu", "tile.cuh", "bucket.cuh", "cluster.cuh", "sieve_internal.cuh", "api.cu"):  # api.cu: the defaults
        f = os.path.join(ROOT, "paper_2310_17746_gb300", "csrc", name)
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel_file: str, key: str = "dram_bytes_per_launch_full"):
    """DRAM bytes (per launch, or the given key) from a committed ncu summary,
    if the kernel sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", kernel_file)
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != source_hash():
        return None
    return d.get(key)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.rows: list[list[str]] = []
        self.proc = None
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid(torch, dev: int):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(target_s: float, steps: int | None = None):
    """Time the oracle on 2^30-number blocks spread across [2, 1e12]."""
    import oracle
    base = oracle.base_table(10**6)
    nblocks_total = WIDTH // SEG_WIDTH
    order = [int(i * 0.6180339887 * nblocks_total) % nblocks_total for i in range(1, 64)]
    width = 0
    spent = 0.0
    times = []
    for n, b in enumerate(order):
        lo = max(2, b * SEG_WIDTH)
        hi = min(WIDTH + 1, (b + 1) * SEG_WIDTH)
        t = time.perf_counter()
        oracle.count_range(lo, hi, base=base)
        dt = time.perf_counter() - t
        times.append((hi - lo, dt))
        width += hi - lo
        spent += dt
        if steps is None and spent >= target_s:
            break
        if steps is not None and n + 1 >= steps:
            break
    return width, spent, times, oracle.default_threads()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # warm-up steps then timed steps, each one 2^30-number block of the workload
    _, _, _, cores = oracle_sample(0, steps=max(args.warmup, 1))
    width, spent, times, cores = oracle_sample(0, steps=args.steps)
    value = width / spent
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * spent / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": "count [2, 1e12] with 2^30-number block histogram",
                   "sample": f"{len(times)} blocks of 2^30 numbers spread over [2, 1e12], one per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{len(times)} x 2^30-number blocks of [2, 1e12]"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm

# ---------------------------------------------------------------- batch and serving legs

def expected_strikes(lo, hi, first: int, primes) -> float:
    """Expected strikes of a 6k+-1 sieve over the queries [lo[i], hi[i]) with
    the primes below `first` presieved: a prime p strikes the class-1 and
    class-5 multiples m >= max(lo, p^2) below hi, one in 3p of the numbers.
    Primes up to sqrt(lo) give w / (3p); those in (sqrt(lo), sqrt(hi)] give
    (hi - p^2) / (3p) = hi / (3p) - p / 3.  Summed with prefix sums of 1/p and
    p over the primes, so that thousands of queries cost a few array passes
    (an expected value: the exact count differs by rounding, < 1 per prime)."""
    import numpy as np
    p = primes[primes >= first].astype(np.float64)
    inv = np.concatenate([[0.0], np.cumsum(1.0 / p)])
    sp = np.concatenate([[0.0], np.cumsum(p)])
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    a = np.searchsorted(p, np.sqrt(lo), side="right")
    b = np.searchsorted(p, np.sqrt(np.maximum(hi - 1, 0)), side="right")
    w = hi - lo
    low = w / 3.0 * inv[a]
    high = hi / 3.0 * (inv[b] - inv[a]) - (sp[b] - sp[a]) / 3.0
    return float(np.sum(low + np.maximum(high, 0.0)))


def naive_leg() -> dict:
    """The plain one-range-per-launch GPU sieve (sieve_range_naive: one bit
    per odd number in global memory, a global atomic AND per multiple, then a
    popcount pass) against the segmented path on the same GPU, for the three
    range workloads: [2, 1e8] as a list, [2, 1e10] and [2, 1e12] as counts.
    Device outputs, CUDA events on the context's stream; the naive call
    allocates its bitmap (62.5 GB at 1e12) inside every call, by design."""
    import numpy as np
    import torch

    from paper_2310_17746_gb300 import binding

    st = torch.cuda.current_stream()

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            fn()
            b.record(st)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    rows = []
    for name, lo, hi, mode, reps in (("[2, 1e8] uint64 list", 2, 10**8 + 1, "list", 3),
                                     ("[2, 1e10] count", 2, 10**10 + 1, "count", 2),
                                     ("[2, 1e12] count", 2, 10**12 + 1, "count", 1)):
        with binding.Sieve(hi) as sv:
            if mode == "list":
                n = sv.range_count(lo, hi).count
                o1 = torch.empty(n, dtype=torch.int64, device="cuda")
                o2 = torch.empty(n, dtype=torch.int64, device="cuda")
                sv.range_list(lo, hi, out=o1)
                sv.naive_list(lo, hi, out=o2)
                assert torch.equal(o1, o2)
                t_seg = timed(lambda: sv.range_list(lo, hi, out=o1), reps)
                t_naive = timed(lambda: sv.naive_list(lo, hi, out=o2), reps)
            else:
                tot = torch.zeros(2, dtype=torch.int64, device="cuda")
                sv.range_count(lo, hi, out=tot)
                ref = sv.naive_count(lo, hi)
                assert (int(tot[0]), int(tot[1]) % 2**64) == (ref.count, ref.checksum)
                t_seg = timed(lambda: sv.range_count(lo, hi, out=tot, asynchronous=True), 3)
                t_naive = timed(lambda: sv.naive_count(lo, hi), reps)
        rows.append({"workload": name, "naive_ms": round(t_naive, 3), "segmented_ms": round(t_seg, 3),
                     "speedup": round(t_naive / t_seg, 1), "naive_numbers_per_s": (hi - lo) / (t_naive / 1e3)})
    return {"comparator": "sieve_range_naive (plain global-bitmap GPU sieve, one range per call)", "configs": rows}


def far_leg(steps: int) -> dict:
    """Far ranges through sieve_range (count, device output): the default
    path (large primes through the bucket sieve) against the same call with
    the bucket sieve off (every prime located in every tile, or, where the
    planner prefers it, the batch path's strips) and through cluster segments
    of 16 CTAs."""
    import torch

    from paper_2310_17746_gb300 import binding

    st = torch.cuda.current_stream()
    rows = []
    for lo, hi in ((10**14, 10**14 + 10**11), (10**16, 10**16 + 10**10), (10**18, 10**18 + 10**9)):
        with binding.Sieve(hi) as sv:
            sv.set_phase_timing(True)
            out = torch.zeros(2, dtype=torch.int64, device="cuda")
            rec = {"range": f"[{lo:.0e}, {lo:.0e} + {hi - lo:.0e})", "width": hi - lo}
            results = []
            # buckets: the default; no_buckets: every prime located in every
            # tile (an asynchronous call never leaves the tile path); strips: a
            # synchronous call with the bucket sieve off, which the planner
            # may send to the batch path (its host planning is inside the events)
            # cluster: the primes above 4 L located once per segment of 16
            # tiles and struck through distributed shared memory (cluster.cuh)
            for name, opts, asy in (("buckets", {}, True), ("no_buckets", {"bucket_threshold": 0}, True),
                                    ("strips_route", {"bucket_threshold": 0}, False),
                                    ("cluster", {"cluster_ctas": 16, "cluster_threshold": 4}, True)):
                sv.set_options(**opts)
                sv.range_count(lo, hi, out=out)
                torch.cuda.synchronize()
                ts = []
                for _ in range(max(2, min(steps, 5))):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(st)
                    sv.range_count(lo, hi, out=out, asynchronous=asy)
                    b.record(st)
                    torch.cuda.synchronize()
                    ts.append(a.elapsed_time(b))
                results.append((int(out[0]), int(out[1])))
                rec[name + "_ms"] = round(min(ts), 3)
                if name == "buckets":
                    rec["bucket_waves"] = int(sv.phase_times()["bucket_waves"])
            assert results[0] == results[1] == results[2] == results[3], (lo, results)
            rec["count"] = results[0][0]
            rec["speedup"] = round(min(rec["no_buckets_ms"], rec["strips_route_ms"]) / rec["buckets_ms"], 2)
            rows.append(rec)
    return {"metric": "sieved range width/s far up (count)", "ranges": rows}


def batch_leg(steps: int, warmup: int) -> dict:
    """Batched range queries/s: the 4096-query workload (seed 0: lo log-uniform
    in [1e6, 1e15], width in [1e3, 1e8], half list mode) in one batched call,
    after the autotuner picked its tunables; against one range launch per query
    on the same GPU; and end to end with host output buffers."""
    import numpy as np
    import torch

    from paper_2310_17746_gb300 import binding, workloads

    q = workloads.batch_queries()
    nq = len(q)
    sv = binding.Sieve(int(q.hi.max()) + 1)
    t0 = time.perf_counter()
    tuned, tuned_ms = sv.autotune_batch(q.lo, q.hi, q.mode, reps=1)
    tune_s = time.perf_counter() - t0
    dev = torch.device("cuda")
    cnt_h, _, _ = sv.range_batch(q.lo, q.hi, np.zeros(nq, np.uint8))
    list_mask = q.mode == workloads.MODE_LIST
    need = int(cnt_h[list_mask, 0].astype(np.int64).sum())
    c = torch.zeros((nq, 2), dtype=torch.int64, device=dev)
    o = torch.zeros(nq + 1, dtype=torch.int64, device=dev)
    v = torch.empty(max(need, 1), dtype=torch.int64, device=dev)
    st = torch.cuda.current_stream(dev)
    launches0 = sv.launch_count()
    for _ in range(max(warmup, 3)):
        sv.range_batch(q.lo, q.hi, q.mode, cnt=c, offsets=o, values=v)
    torch.cuda.synchronize()
    ts = []
    launches1 = sv.launch_count()
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        sv.range_batch(q.lo, q.hi, q.mode, cnt=c, offsets=o, values=v)
        b.record(st)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / 1e3)
    per_call_launches = (sv.launch_count() - launches1) / steps
    got = c.cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, cnt_h), "batched list run disagrees with the count-only run"
    t_dev = statistics.mean(ts)
    # one range launch per query (same outputs, device memory)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sv.range_batch(q.lo, q.hi, q.mode, cnt=c, offsets=o, values=v, naive=True)
    torch.cuda.synchronize()
    t_naive = time.perf_counter() - t0
    # end to end with host buffers (pinned, so the copies run at full speed)
    hc = torch.zeros((nq, 2), dtype=torch.int64).pin_memory().numpy()
    ho = torch.zeros(nq + 1, dtype=torch.int64).pin_memory().numpy()
    hv = torch.empty(max(need, 1), dtype=torch.int64).pin_memory().numpy()
    sv.range_batch(q.lo, q.hi, q.mode, cnt=hc, offsets=ho, values=hv)
    te = []
    for _ in range(max(1, min(steps, 3))):
        t0 = time.perf_counter()
        sv.range_batch(q.lo, q.hi, q.mode, cnt=hc, offsets=ho, values=hv)
        te.append(time.perf_counter() - t0)
    opts = sv.options()
    sv.close()
    # roofline: the batch's strikes (expected, see expected_strikes) over its
    # device time, against the shared-memory atomic-AND rate every strike
    # uses; and its list bytes against HBM
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    atom_cf, _ = binding.measure_smem_atomics(torch.cuda.current_device())
    first = LAST_PRESIEVED[opts["presieve_groups"]] + 1
    strikes = expected_strikes(q.lo, q.hi, first, small_primes(int(math.isqrt(int(q.hi.max())))))
    atom_peak = props.multi_processor_count * atom_cf * sm_max * 1e6 / 1e9
    hbm_peak = float(peaks.get("hbm_gbs") or 6800.0)
    return {
        "metric": "batched range queries/s", "value": nq / t_dev, "unit": "queries/s",
        "roofline": {"bound": "alu", "resource": "shared-memory atomic AND lane operations (the strikes)",
                     "achieved": strikes / t_dev / 1e9, "peak": atom_peak, "unit": "Gop/s",
                     "frac": strikes / t_dev / 1e9 / atom_peak, "traffic": None,
                     "strikes_per_batch": strikes,
                     "peak_basis": f"measured (sieve_measure_smem_atomics): {atom_cf:.2f} lane-ops/clk/SM x "
                                   f"{props.multi_processor_count} SMs x {sm_max:.0f} MHz",
                     "list_bytes_roofline": {"bound": "hbm", "achieved": need * 8 / t_dev / 1e9, "peak": hbm_peak,
                                             "unit": "GB/s", "frac": need * 8 / t_dev / 1e9 / hbm_peak}},
        "ms_per_batch": 1e3 * t_dev, "queries": nq, "list_primes": need,
        "workload": "4096 queries, seed 0: lo = floor(10^U(6,15)), width = floor(10^U(3,8)), half list mode "
                    "(uint64 primes, CSR), base primes <= 3.2e7 on the device",
        "naive_one_launch_per_query": {"value": nq / t_naive, "unit": "queries/s", "ms": 1e3 * t_naive},
        "speedup_vs_naive": t_naive / t_dev,
        "e2e": {"value": nq / statistics.mean(te), "unit": "queries/s",
                "h2d_bytes_per_step": int(nq * 17), "d2h_bytes_per_step": int(nq * 16 + (nq + 1) * 8 + need * 8)},
        "list_write_gbs": need * 8 / t_dev / 1e9,
        "autotuned": {k: tuned[k] for k in ("batch_tile_bits", "block_threads", "chunk_primes", "presieve_groups")},
        "autotune_s": tune_s, "kernels_per_call": per_call_launches,
        "l2": "outputs (6 GB of primes) exceed L2; no flush",
    }


def list_leg(steps: int, warmup: int) -> dict:
    """The list path: the uint64 primes of [1e12, 1e12 + 2e10) written into a
    device buffer through sieve_range, two-pass (default: tile kernel writes
    bitmaps, scan, compaction) and single-pass (each tile compacted from
    shared memory at an offset found by look-back).  Roofline: the 8 bytes
    per listed prime the method must write, over the whole call, against the
    measured copy bandwidth; the compaction kernel's own rate beside it."""
    import numpy as np
    import torch

    from paper_2310_17746_gb300 import binding

    lo, hi = 10**12, 10**12 + 2 * 10**10
    sv = binding.Sieve(hi)
    n = sv.range_count(lo, hi).count
    out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    sv.set_phase_timing(True)
    st = torch.cuda.current_stream()
    res = {}
    for sp in (0, 1):
        sv.set_options(list_single_pass=sp)
        for _ in range(max(1, warmup)):
            sv.range_list(lo, hi, out=out)
        calls, phases = [], []
        for _ in range(steps):
            s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            s_.record(st)
            got = sv.range_list(lo, hi, out=out)
            e_.record(st)
            torch.cuda.synchronize()
            calls.append(s_.elapsed_time(e_) / 1e3)
            phases.append(sv.phase_times())
            assert got == n, (got, n)
        head = out[:4].cpu().numpy()
        tail = out[n - 2:n].cpu().numpy()
        assert head[0] == 1000000000039 and (np.diff(head) > 0).all() and tail[-1] < hi, (head, tail)
        res[sp] = (statistics.mean(calls), phases)
    sv.close()
    t_call, phases = res[0]
    ph = phases[-1]
    compact_s = statistics.mean(p["compact_ms"] for p in phases) / 1e3
    sieve_s = statistics.mean(p["sieve_ms"] for p in phases) / 1e3
    bitmap_bytes = int(ph["tiles"]) * (int(ph["tile_len"]) // 32) * 8
    peaks = measured_peaks()
    peak = float(peaks.get("hbm_gbs") or 6800.0)
    alg_bytes = n * 8
    achieved = alg_bytes / t_call / 1e9
    per_prime = profiled_traffic("compact_kernel_list_1e12.json", "dram_bytes_per_listed_prime")
    return {
        "metric": "listed primes/s", "value": n / t_call, "unit": "primes/s",
        "workload": "the uint64 primes of [1e12, 1e12 + 2e10) into a device buffer (sieve_range, list mode)",
        "primes": n, "ms_per_call": 1e3 * t_call,
        "tile_kernel_ms": 1e3 * sieve_s, "compaction_ms": 1e3 * compact_s,
        "single_pass_ms_per_call": 1e3 * res[1][0],
        "roofline": {"bound": "hbm", "kernel": "range_tiles_kernel + compact_kernel (whole call)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": per_prime * n if per_prime else None, "algorithmic_bytes": alg_bytes,
                     "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json)" if peaks.get("hbm_gbs")
                     else "fallback 6.8 TB/s",
                     "compaction_kernel_gbs": (alg_bytes + bitmap_bytes) / compact_s / 1e9},
        "l2": "output (5.8 GB) exceeds L2; no flush",
    }


def serving_leg(rates=(1000, 3000, 10000, 30000, 100000), seconds: float = 1.0, max_n: int = 10000) -> dict:
    """Open-loop Poisson request streams (seed 1: lo log-uniform in [1e6, 1e18],
    width in [1e3, 1e9], 20% list mode) against the continuous-batching server;
    latency = submit to result ready on the server.  Results are collected into
    device memory.  Compared, at every offered rate and with the same requests,
    with one range launch per request in arrival order."""
    import threading as th

    import numpy as np
    import torch

    from paper_2310_17746_gb300 import binding, workloads

    dev = torch.device("cuda")
    sv = binding.Sieve(10**18 + 10**9 + 1)  # base primes <= 1e9 on the device
    # the batch tunables for this workload: autotuned on 512 requests of the
    # same distribution drawn with another seed (not the measured ones)
    sample = workloads.serving_arrivals(1000.0, 512, seed=7).queries
    t0 = time.perf_counter()
    tuned, tuned_ms = sv.autotune_batch(sample.lo, sample.hi, sample.mode, reps=1)
    tune_s = time.perf_counter() - t0
    scratch = torch.empty(1 << 27, dtype=torch.int64, device=dev)  # 1 GiB landing zone for lists
    out = {"workload": "Poisson arrivals, seed 1: lo = floor(10^U(6,18)), width = floor(10^U(3,9)), "
                       "list with probability 0.2; base primes <= 1e9 on the device", "rates": [],
           "autotuned": {"options": {k: tuned[k] for k in ("batch_tile_bits", "block_threads", "chunk_primes", "presieve_groups")},
                         "sample": "512 requests of the serving distribution, seed 7", "sample_ms": tuned_ms,
                         "seconds": tune_s}}
    srv = binding.Server(sv, pool_bytes=32 << 30)
    def drain(expected: int, timeout_s: float) -> int:
        """Collect finished requests until `expected` were collected."""
        got, t_end = 0, time.perf_counter() + timeout_s
        while got < expected and time.perf_counter() < t_end:
            rid = srv.next_done(timeout_us=2000)
            if rid is not None:
                got += srv.poll(rid, out=scratch) is not None
        return got

    # warm-up: every tile width and the strip path
    warm = workloads.serving_arrivals(1000.0, 200, seed=99)
    ids = [srv.submit(int(a), int(b), int(m)) for a, b, m in zip(warm.queries.lo, warm.queries.hi, warm.queries.mode)]
    drain(len(ids), 120.0)
    srv.stats(reset=True)
    for rate in rates:
        n = int(min(max_n, rate * seconds))
        arr = workloads.serving_arrivals(float(rate), n, seed=1)
        lo, hi, mode = arr.queries.lo.tolist(), arr.queries.hi.tolist(), arr.queries.mode.tolist()
        t_arr = arr.t_arrive.tolist()
        admitted = [0]
        rejected = [0]
        done_flag = [False]
        collected = [0]

        def collector():
            while not done_flag[0] or collected[0] < admitted[0]:
                rid = srv.next_done(timeout_us=2000)
                if rid is not None:
                    collected[0] += srv.poll(rid, out=scratch) is not None
                elif done_flag[0] and time.perf_counter() - t0 > t_limit:
                    return

        t_limit = seconds * 20 + 30
        t0 = time.perf_counter()
        col = th.Thread(target=collector)
        col.start()
        for i in range(n):
            while time.perf_counter() - t0 < t_arr[i]:
                pass
            if srv.try_submit(lo[i], hi[i], mode[i]) is None:
                rejected[0] += 1
            else:
                admitted[0] += 1
        t_sub = time.perf_counter() - t0
        done_flag[0] = True
        col.join()
        t_end = time.perf_counter() - t0
        st = srv.stats(reset=True)
        out["rates"].append({
            "offered_per_s": rate, "requests": n, "admitted": admitted[0], "rejected_busy": rejected[0],
            "completed": collected[0], "queries_per_s": collected[0] / t_end, "submit_s": t_sub, "p50_us": st["p50_us"],
            "p99_us": st["p99_us"], "mean_us": st["mean_us"], "max_us": st["max_us"],
            "batches": st["batches"], "mean_batch": st["mean_batch"], "overlapped_batches": st["overlapped_batches"]})
    srv.stop()
    # one range launch per request, in arrival order, same requests at every rate
    naive = []
    for rate in rates:
        n = int(min(max_n, rate * seconds))
        arr = workloads.serving_arrivals(float(rate), n, seed=1)
        lat = []
        t0 = time.perf_counter()
        for i in range(n):
            while time.perf_counter() - t0 < arr.t_arrive[i]:
                pass
            a, b, m = int(arr.queries.lo[i]), int(arr.queries.hi[i]), int(arr.queries.mode[i])
            if m == workloads.MODE_LIST:
                sv.range_list(a, b, out=scratch)
            else:
                sv.range_count(a, b)
            lat.append(time.perf_counter() - t0 - arr.t_arrive[i])
        t_end = time.perf_counter() - t0
        lat.sort()
        naive.append({"offered_per_s": rate, "requests": n, "queries_per_s": n / t_end,
                      "p50_us": 1e6 * lat[len(lat) // 2], "p99_us": 1e6 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]})
    out["naive_one_launch_per_query"] = naive
    sv.close()
    return out


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2310_17746_gb300 import binding

    rank, world, local = dist_env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    lo, hi = rank_range(rank)
    stream = torch.cuda.current_stream(dev)
    sv = binding.Sieve(hi, device=local, stream=stream.cuda_stream)
    # the tunables: from the tuning cache for this device and workload, or
    # tuned now on a 2e10-wide sample of the range (and stored by rank 0)
    t0 = time.perf_counter()
    got = sv.tune_cache_load(TUNE_CACHE, TUNE_WORKLOAD)
    if got is None:
        mid = lo + (hi - lo) // 2
        tuned, tuned_ms = sv.autotune_range(mid, mid + 2 * 10**10, reps=2)
        tune_source = "tuned in this run on [mid, mid + 2e10) of the range"
        if rank == 0:
            sv.tune_cache_store(TUNE_CACHE, TUNE_WORKLOAD, tuned_ms)
    else:
        tuned, tuned_ms = got
        tune_source = "tuning cache " + os.path.relpath(TUNE_CACHE, ROOT)
    tune_s = time.perf_counter() - t0
    nb = binding.Sieve.nbins(lo, hi, SEG_WIDTH)
    counts = torch.zeros(nb, dtype=torch.int64, device=dev)
    total = torch.zeros(2, dtype=torch.int64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MiB > L2

    def step():
        sv.segment_counts(lo, hi, SEG_WIDTH, counts=counts, total=total, asynchronous=True)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert rank != 0 or int(total[0]) == PI_1E12, f"pi(1e12) mismatch: {int(total[0])}"

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(gpu_uuid(torch, local))
    barrier()
    torch.cuda.synchronize()
    launches0 = sv.launch_count()
    clocks.start()
    time.sleep(0.25)  # first sample lands inside the timed region
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i)  # evict L2 between steps, outside the timed events
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier()
    clk = clocks.stop()
    launches = sv.launch_count() - launches0
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_local = sum(step_ms) / 1e3
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    widths = sum((rank_range(r)[1] - rank_range(r)[0]) for r in range(world))
    value = widths * args.steps / t_max
    got_count = int(total[0])

    # end to end through the C ABI with host buffers (copies inside the timed region)
    host_counts = np.zeros(nb, dtype=np.uint64)
    e2e_times = []
    for i in range(min(args.steps, 3)):
        flush.fill_(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tot_host, _ = sv.segment_counts(lo, hi, SEG_WIDTH, counts=host_counts)
        e2e_times.append(time.perf_counter() - t0)
    assert rank != 0 or tot_host.count == PI_1E12
    e2e_local = statistics.mean(e2e_times)
    te = torch.tensor([e2e_local], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = widths / float(te.item())

    if rank != 0:
        sv.close()
        if world > 1:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel (the tile sieve; one launch per step):
    # its strikes are shared-memory atomic ANDs, whose throughput on this
    # device is measured live (conflict-free lanes per SM per clock)
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0)
    opts = sv.options()
    first = LAST_PRESIEVED[opts["presieve_groups"]] + 1
    alg = algorithmic_ops(lo, hi, first)
    per_launch_s = t_local / args.steps
    atom_cf, atom_rand = binding.measure_smem_atomics(local)
    achieved = alg["strikes"] / per_launch_s / 1e9
    peak = props.multi_processor_count * atom_cf * sm_max * 1e6 / 1e9
    traffic = profiled_traffic("range_tiles_count_1e12.json")

    batch = serving = listing = naive = far = None
    if world == 1 and not args.no_naive:
        naive = naive_leg()
    if world == 1 and not args.no_far:
        far = far_leg(args.steps)
    if world == 1 and not args.no_batch:
        batch = batch_leg(args.steps, args.warmup)
    if world == 1 and not args.no_list:
        listing = list_leg(args.steps, args.warmup)
    if world == 1 and not args.no_serving:
        serving = serving_leg()

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        w, spent, times, cores = oracle_sample(args.cpu_seconds)
        cpu = {"value": w / spent, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{len(times)} blocks of 2^30 numbers spread over [2, 1e12] ({w:.3e} numbers, {spent:.1f} s)"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "count [2, 1e12] with 2^30-number block histogram (932 bins); "
                               "rank r>0 sieves the next contiguous range of rank 0's modelled cost",
                   "lo": lo, "hi_exclusive": hi, "seg_width": SEG_WIDTH,
                   "tile_bits": opts["tile_bits"], "block_threads": opts["block_threads"],
                   "group_hits": opts["group_hits"],
                   "autotuned": {"options": {k: opts[k] for k in ("tile_bits", "block_threads", "ctas_per_sm",
                                                                  "group_hits", "presieve_groups",
                                                                  "bucket_threshold")},
                                 "source": tune_source, "tuned_sample_ms": tuned_ms, "seconds": tune_s},
                   "l2": "flushed between steps (256 MiB write outside the timed events)"},
        "check": {"pi_1e12": got_count, "expected": PI_1E12, "ok": got_count == PI_1E12},
        "roofline": {"bound": "alu", "resource": "shared-memory atomic AND lane operations (the strikes)",
                     "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "range_tiles_kernel",
                     "strikes_per_launch": alg["strikes"], "candidate_words_per_launch": alg["candidate_words"],
                     "peak_basis": f"measured (sieve_measure_smem_atomics, live): {atom_cf:.2f} conflict-free "
                                   f"lane-ops/clk/SM ({atom_rand:.2f} at random banks) x "
                                   f"{props.multi_processor_count} SMs x {sm_max:.0f} MHz "
                                   f"({'measured' if peaks else 'fallback'} max SM clock)",
                     "peak_nominal_smem": props.multi_processor_count * 32 * sm_max * 1e6 / 1e9},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 16,
                "d2h_bytes_per_step": 8 * nb + 16},
        "gpu_launches": launches,
        "naive_gpu": (None if naive is None else
                      {"value": naive["configs"][-1]["naive_numbers_per_s"], "unit": UNIT,
                       "ms": naive["configs"][-1]["naive_ms"],
                       "headline_speedup": (naive["configs"][-1]["naive_ms"] / (1e3 * t_max / args.steps)),
                       "all": naive}),
        "far": far,
        "batch": batch,
        "list": listing,
        "serving": serving,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    print(json.dumps(line), flush=True)
    sv.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
