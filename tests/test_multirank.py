"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank runs its own
independent simulation (distinct seeds, same sizes), the timed region is reduced with
a max over ranks, and the whole-job throughput counts all ranks' cycles."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]
    mx = bench.reduce_max(ms, dist, None)
    w = bench.workload(32, rank)
    out[rank] = (mx, bench.weak_throughput(10, world, mx), w.seed, w.Nz, w.Nr)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_weak_throughput():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 150.0                      # max over ranks on every rank
    assert r0[1] == pytest.approx(2 * 10 / 0.150)       # both ranks' cycles in the job total
    assert r0[2] != r1[2] and (r0[3], r0[4]) == (r1[3], r1[4])   # independent sims, same size


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.weak_throughput(60, 1, 750.0) == pytest.approx(80.0)
