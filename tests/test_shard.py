"""Multi-rank timing and sharding logic on CPU with the gloo backend
(world size 2): no GPU, no data-path collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2401_14221_gb300 import shard


def test_shard_ranges_cover_everything_once():
    for n in (0, 1, 7, 960000, 960001):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard.shard_range(n, r, world)
                seen.extend(range(lo, hi)) if n < 100 else seen.append((lo, hi))
            if n < 100:
                assert seen == list(range(n))
            else:
                assert seen[0][0] == 0 and seen[-1][1] == n
                assert all(a[1] == b[0] for a, b in zip(seen, seen[1:]))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shard.barrier(world)
        elapsed = 1.0 + rank  # rank 1 is the slow one
        m = shard.max_over_ranks(elapsed, world)
        value = shard.whole_job_throughput(960000, 10, world, m)
        out[rank] = (m, value, shard.rank_seed(1, rank))
        shard.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert out[0][0] == out[1][0] == 2.0
    assert out[0][1] == pytest.approx(2 * 960000 * 10 / 2.0)
    assert out[0][2] != out[1][2]
