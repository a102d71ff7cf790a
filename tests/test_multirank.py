"""The N > 1 path of bench.py (independent replicas per rank, no data-path
collective): barrier and max-over-ranks timing and the whole-job PID, run as
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    t = [0.8, 1.3][rank]  # per-rank wall seconds of the timed region
    tmax = bench.max_over_ranks(t, dist, "cpu")
    pid = bench.whole_job_pid(tmax, steps=10, dof_per_rank=1000, world=world)
    q.put((rank, tmax, pid, bench.dist_env()))
    dist.destroy_process_group()


def test_two_rank_timing_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, pid, env in res:
        assert tmax == 1.3  # every rank reports the slowest replica
        assert abs(pid - 1.3e9 / (10 * 5 * 1000 * 2)) < 1e-9 * pid  # all ranks' DOF in the denominator
        assert env == (2, rank, 0)
