"""The sharded path driven by the CUDA library: one range split over 2 gloo
ranks (processes) that share the one GPU, each sieving its contiguous shard
through its own library context, reduced with torch.distributed.  The result
must equal the unsharded GPU run and the CPU oracle exactly (count, checksum
mod 2^64, per-segment counts, and the concatenated list)."""
import os
import socket

import numpy as np
import pytest

from paper_2310_17746_gb300 import shard

pytestmark = pytest.mark.gpu

LO, HI, W = 2, 10**10 + 1, 1 << 24
LLO, LHI = 10**12 - 3_000_000, 10**12 + 7_000_001


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_2310_17746_gb300 import binding

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()  # each rank on its own stream of the shared GPU
        with torch.cuda.stream(stream), binding.Sieve(LHI, device=0, stream=stream.cuda_stream) as sv:
            def count_fn(a, b, w):
                tot, bins = sv.segment_counts(a, b, w)
                return tot.count, tot.checksum, bins
            c, s, bins = shard.distributed_segment_counts(count_fn, LO, HI, W)
            lst = shard.distributed_list(lambda a, b: sv.range_list(a, b), LLO, LHI)
        out.put((rank, c, s, bins.tobytes(), lst.tobytes()))
    finally:
        dist.destroy_process_group()


def test_sharded_cuda_equals_unsharded_and_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as tmp

    import oracle
    from paper_2310_17746_gb300 import binding

    world = 2
    ctx = tmp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    with binding.Sieve(LHI) as sv:
        tot, gbins = sv.segment_counts(LO, HI, W)
        glist = sv.range_list(LLO, LHI)
    oc, osum, obins = oracle.segment_counts(LO, HI, W)
    assert (tot.count, tot.checksum) == (oc, osum)
    np.testing.assert_array_equal(gbins, obins)
    np.testing.assert_array_equal(glist, oracle.list_range(LLO, LHI))
    for rank, c, s, bins, lst in res:
        assert (c, s) == (oc, osum), rank
        np.testing.assert_array_equal(np.frombuffer(bins, dtype=np.uint64), obins)
        np.testing.assert_array_equal(np.frombuffer(lst, dtype=np.uint64), glist)
