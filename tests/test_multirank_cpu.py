"""Multi-rank host logic on two gloo ranks on CPU (rendezvous on 127.0.0.1).
The benchmark's multi-GPU path is replicas with no data-path collective:
each rank solves its own batch and only the timing is reduced (max over
ranks).  A batch of RANSAC problems is split over ranks as contiguous,
cost-balanced ranges (api.shard_ranges); each rank runs its range with
problem_base = its start, and the gathered results equal one run over all
problems (checked with the FP64 oracle standing in for each rank's work)."""
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


def _shard_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import workloads
    from paper_2402_18008_gb300 import api
    rb = workloads.ransac_batch(P=24, seed=13, n_max=1500, cap=256)
    N = np.diff(rb.offsets)
    a, b = api.shard_ranges(N * rb.n_hyp, world)[rank]
    lo, hi = int(rb.offsets[a]), int(rb.offsets[b])
    r = oracle.ransac(rb.corr[lo:hi], rb.offsets[a:b + 1] - lo, rb.n_hyp[a:b], 3.0, 5, problem_base=a, want_mask=True)
    part = (a, b, r["best_hyp"], r["best_count"], r["best_H"], r["hyp_counts"], r["inlier_mask"])
    parts = [None] * world
    dist.all_gather_object(parts, part)
    if rank == 0:
        q.put(parts)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_a_ransac_batch_by_cost():
    import numpy as np
    import oracle
    import workloads
    from paper_2402_18008_gb300 import api
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rb = workloads.ransac_batch(P=24, seed=13, n_max=1500, cap=256)
    one = oracle.ransac(rb.corr, rb.offsets, rb.n_hyp, 3.0, 5, want_mask=True)
    assert [(a, b) for a, b, *_ in parts] == [(0, parts[0][1]), (parts[0][1], 24)]
    assert np.array_equal(np.concatenate([p[2] for p in parts]), one["best_hyp"])
    assert np.array_equal(np.concatenate([p[3] for p in parts]), one["best_count"])
    assert np.array_equal(np.concatenate([p[4] for p in parts]), one["best_H"])
    assert np.array_equal(np.concatenate([p[5] for p in parts]), one["hyp_counts"])
    assert np.array_equal(np.concatenate([p[6] for p in parts]), one["inlier_mask"])
    # each range's cost lies within one problem's cost of the mean
    cost = np.diff(rb.offsets) * rb.n_hyp
    per = np.array([cost[a:b].sum() for a, b, *_ in parts])
    assert np.all(np.abs(per - cost.sum() / 2) <= cost.max())


def test_shard_ranges_cover_every_problem_once_and_balance_the_cost():
    import numpy as np
    from paper_2402_18008_gb300 import api
    rng = np.random.default_rng(2)
    for world in (1, 2, 3, 8):
        for P in (1, 5, 37, 512):
            c = rng.integers(0, 1000, P).astype(float)
            r = api.shard_ranges(c, world)
            assert len(r) == world and r[0][0] == 0 and r[-1][1] == P
            assert all(r[i][1] == r[i + 1][0] and r[i][0] <= r[i][1] for i in range(world - 1))
            loads = np.array([c[a:b].sum() for a, b in r])
            assert np.all(np.abs(loads - c.sum() / world) <= c.max() + 1e-9)
    assert api.shard_ranges([0, 0, 0], 2)[-1][1] == 3


def test_single_process_helpers_without_a_process_group():
    import torch
    import bench
    assert bench.max_over_ranks(3.0, torch, torch.device("cpu")) == 3.0
    assert bench.job_throughput(1 << 26, 1, 1.0) == pytest.approx(6.7108864e10)
