"""The multi-GPU path of the benchmark is replicas with no data-path
collective: each rank solves its own batch and only the timing is reduced
(max over ranks).  This checks that host-side logic with two gloo ranks on
CPU (rendezvous on 127.0.0.1)."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads
    my_ms = 1.5 + rank                     # a slower rank 1
    slowest = bench.max_over_ranks(my_ms, torch, torch.device("cpu"))
    seed = bench.rank_seed(rank)
    sets = workloads.minimal_sets(64, seed=seed, keep_truth=False)
    q.put((rank, slowest, seed, sets.pts[:, :4].copy(), bench.job_throughput(64, world, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in range(2):
        r, slowest, seed, head, thr = q.get(timeout=120)
        got[r] = (slowest, seed, head, thr)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0][0] == got[1][0] == 2.5          # both ranks report the slowest time
    assert got[0][1] != got[1][1]                  # different seeds: different batches
    assert not (got[0][2] == got[1][2]).all()
    assert got[0][3] == got[1][3] == pytest.approx(2 * 64 / 2.5e-3)


def test_single_process_helpers_without_a_process_group():
    import torch
    import bench
    assert bench.max_over_ranks(3.0, torch, torch.device("cpu")) == 3.0
    assert bench.job_throughput(1 << 26, 1, 1.0) == pytest.approx(6.7108864e10)
