"""The multi-rank path of bench.py on the CPU: two gloo ranks (127.0.0.1), one independent
instance per rank.  Checks the max-over-ranks timing, the whole-job value and that only
rank 0 runs the reference arm (the other ranks exit without work)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 100 ms for 1000 units: the job time is the slowest rank's
        tot_ms = bench.max_over_ranks((rank + 1) * 100.0, world)
        value = bench.whole_job_rate(world, 1000, tot_ms)
        dist.barrier()
        ref = bench.run_reference(None, rank, world) if rank != 0 else "skipped"
        out.put((rank, tot_ms, value, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(out.get(timeout=5) for _ in range(world))
    for rank, tot_ms, value, ref in res:
        assert tot_ms == 200.0                      # max over ranks, seen by every rank
        assert value == pytest.approx(2 * 1000 / 0.2)
    assert res[1][3] is None                        # rank 1 returns from the reference arm at once


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 500, 250.0) == pytest.approx(2000.0)
