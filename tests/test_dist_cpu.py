"""Multi-rank host logic of bench.py on CPU with the gloo backend (world size 2).

With --gpus N every rank runs an independent replica of the workload; the only
collective is the timing reduction (maximum over ranks), and the whole-job rate is
all replicas' units divided by the slowest rank's time."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    per_rank = [10.0 + 5.0 * rank, 12.0 - rank]  # (step ms, e2e ms) measured on this rank
    step_ms, e2e_ms = bench.max_over_ranks(per_rank, world)
    rate = bench.whole_job_rate(4.0e10, world, step_ms)
    q.put((rank, step_ms, e2e_ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, step_ms, e2e_ms, rate in out:
        assert step_ms == 15.0 and e2e_ms == 12.0
        assert rate == pytest.approx(2 * 4.0e10 / 15e-3)


def test_single_rank_needs_no_collective():
    import bench

    assert bench.max_over_ranks([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.whole_job_rate(100.0, 1, 1000.0) == pytest.approx(100.0)
