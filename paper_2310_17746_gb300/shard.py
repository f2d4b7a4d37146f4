"""Sharding one range over ranks (one process per GPU) and reducing the results.

A range [lo, hi) splits into contiguous value intervals, one per rank, that
are sieved independently (Sections 2.2-2.3: each worker owns a contiguous
chunk; no data crosses between chunks).  The only exchange is the final
reduction: counts, checksums (sums mod 2^64) and per-segment counts add up,
and lists concatenate in rank order because the shards are in value order.

The local sieve is passed in as a function, so the same logic runs over the
CUDA library on GPU ranks and over any other implementation on CPU ranks.
Sums use int64 tensors: two's-complement addition wraps exactly like uint64
addition modulo 2^64, so the checksum survives the all-reduce bit for bit.
"""
from __future__ import annotations

import numpy as np


# Device time of a count per 1e11 numbers at height x, in ms: linear in the
# number of base primes below sqrt(x), each located in every tile; fitted on
# one GB300 to windows of 1e11 from 1e11 to 2e13 (15.4 ... 33.3 ms, within
# 1 %).  Only ratios matter for balancing.
COST_A_MS, COST_B_MS = 13.58, 6.27e-5
_PI_EXACT = 10**7
_pi_table = None


def _pi(y: np.ndarray) -> np.ndarray:
    """pi(y): exact up to 1e7 (a small sieve), y / (ln y - 1) above."""
    global _pi_table
    if _pi_table is None:
        f = np.ones(_PI_EXACT + 1, dtype=bool)
        f[:2] = False
        for i in range(2, int(_PI_EXACT**0.5) + 1):
            if f[i]:
                f[i * i::i] = False
        _pi_table = np.cumsum(f, dtype=np.int32)  # pi(1e7) = 664579
    y = np.asarray(y, dtype=np.float64)
    small = y <= _PI_EXACT
    out = np.empty_like(y)
    out[small] = _pi_table[y[small].astype(np.int64)]
    big = ~small
    out[big] = y[big] / (np.log(y[big]) - 1.0)
    return out


def cost_ms(lo: int, hi: int, steps: int = 2048) -> float:
    """Modelled count time of [lo, hi) in ms (midpoint rule over the density)."""
    if hi <= lo:
        return 0.0
    x = lo + (np.arange(steps) + 0.5) * ((hi - lo) / steps)
    return float(np.sum(COST_A_MS + COST_B_MS * _pi(np.sqrt(x))) * (hi - lo) / steps / 1e11)


def shard_bounds(lo: int, hi: int, world: int, align: int = 6, balance: bool = True) -> list[int]:
    """world + 1 increasing boundaries b[0] = lo <= ... <= b[world] = hi; rank r
    sieves [b[r], b[r+1]).  Inner boundaries are multiples of `align` (tile
    and residue-class friendly).  With balance, each rank gets an equal share
    of the modelled count time (cost_ms): the work per number grows with the
    base primes every tile locates, 1.8 times from 1e12 to 2e13, so equal
    widths would leave the top ranks behind; without, the widths are equal."""
    if world < 1 or hi < lo:
        raise ValueError("need world >= 1 and lo <= hi")
    total = cost_ms(lo, hi) if balance else 0.0
    b = [lo]
    for r in range(1, world):
        if balance and total > 0:
            a, z = b[-1], hi  # the smallest x with cost(lo, x) >= r / world of the total
            want = total * r / world
            while z - a > align:
                m = a + (z - a) // 2
                if cost_ms(lo, m) < want:
                    a = m
                else:
                    z = m
            x = z
        else:
            x = lo + (hi - lo) * r // world
        x = min(max(x - x % align, b[-1]), hi)
        b.append(x)
    b.append(hi)
    return b


def _wrap64(x: int) -> int:
    """A value mod 2^64 as the signed int64 with the same bits."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= 1 << 63 else x


def reduce_count(count: int, checksum: int, bins, group=None):
    """All-reduce (sum) of one rank's count, checksum and per-segment counts
    (a uint64 array in the GLOBAL segment numbering, zero outside the rank's
    shard).  Returns (count, checksum mod 2^64, bins as uint64)."""
    import torch
    import torch.distributed as dist

    nb = 0 if bins is None else int(np.asarray(bins).size)
    t = torch.zeros(2 + nb, dtype=torch.int64)
    t[0] = _wrap64(count)
    t[1] = _wrap64(checksum)
    if nb:
        t[2:] = torch.from_numpy(np.asarray(bins, dtype=np.uint64).view(np.int64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    out = t.numpy().view(np.uint64)
    return int(out[0]), int(out[1]), (out[2:].copy() if nb else None)


def gather_list(local: np.ndarray, group=None) -> np.ndarray:
    """Concatenate every rank's (increasing) list in rank order."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n = torch.tensor([int(local.size)], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    cap = max(sizes + [1])
    buf = torch.zeros(cap, dtype=torch.int64)
    buf[: local.size] = torch.from_numpy(np.asarray(local, dtype=np.uint64).view(np.int64))
    parts = [torch.zeros(cap, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return np.concatenate([p.numpy()[:s].view(np.uint64) for p, s in zip(parts, sizes)])


def distributed_segment_counts(local_fn, lo: int, hi: int, seg_width: int, group=None):
    """Count, checksum and per-segment counts of [lo, hi) over all ranks.

    local_fn(a, b, seg_width) -> (count, checksum, bins) sieves [a, b) on this
    rank, bins numbered from a // seg_width.  Returns the global result on
    every rank."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    b = shard_bounds(lo, hi, world)
    a, e = b[rank], b[rank + 1]
    nb = 0 if hi <= lo else (hi - 1) // seg_width - lo // seg_width + 1
    glob = np.zeros(nb, dtype=np.uint64)
    c = s = 0
    if e > a:
        c, s, bins = local_fn(a, e, seg_width)
        first = a // seg_width - lo // seg_width
        glob[first:first + len(bins)] += np.asarray(bins, dtype=np.uint64)
    return reduce_count(c, s, glob, group)


def distributed_list(local_fn, lo: int, hi: int, group=None) -> np.ndarray:
    """The primes of [lo, hi) gathered from all ranks, increasing.
    local_fn(a, b) -> increasing uint64 array of the primes in [a, b)."""
    import torch.distributed as dist

    rank, world = dist.get_rank(group), dist.get_world_size(group)
    b = shard_bounds(lo, hi, world)
    local = local_fn(b[rank], b[rank + 1]) if b[rank + 1] > b[rank] else np.zeros(0, np.uint64)
    return gather_list(np.asarray(local, dtype=np.uint64), group)
