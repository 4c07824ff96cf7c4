"""The N > 1 path on CPU ranks (gloo, world size 2): slices are sharded with no
data-path collective, the timing is the maximum over ranks, and the within-slice
view sharding (not built on the GPU: one GPU per run) is exact — the sum over
ranks of the backprojections of each rank's views equals the full A^T, and the
ranks' projections are the full A's rows (Eq. 1 is a sum over views' rays)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # slices: every rank solves its own, with seeds no other rank uses
        ws = bench.workloads(6, rank)
        seeds = torch.tensor([w.seed for w in ws])
        every = [torch.zeros_like(seeds) for _ in range(world)]
        dist.all_gather(every, seeds)
        sets = [set(e.tolist()) for e in every]     # (a rank's 800- and 200-view slices share a seed)
        assert all(sets[a].isdisjoint(sets[b]) for a in range(world) for b in range(a + 1, world))
        # timing: the job's time is the slowest rank's
        t = bench.max_over_ranks([10.0 + rank, 5.0 - rank], dist, "cpu")
        assert t == [10.0 + world - 1, 5.0]
        # view sharding of one slice: rank r takes views [r V/w, (r+1) V/w)
        V, n, nb = 12, 20, 29
        full = oracle.Geometry(n, 1.3, V, nb, beta0=0.2)
        dg = 2.0 * np.arcsin(n * 1.3 / np.sqrt(2.0) / full.dso_mm) / nb
        full = oracle.Geometry(n, 1.3, V, nb, dgamma=dg, beta0=0.2)
        vr = V // world
        part = oracle.Geometry(n, 1.3, vr, nb, dgamma=dg, beta0=0.2 + full.arc * rank / world,
                               arc=full.arc / world)
        rng = np.random.Generator(np.random.PCG64(5))
        Y = rng.standard_normal((V, nb))
        X = rng.standard_normal((n, n))
        mine = torch.from_numpy(np.ascontiguousarray(oracle.backproject(part, Y[rank * vr:(rank + 1) * vr])))
        dist.all_reduce(mine)
        ref = oracle.backproject(full, Y)
        assert np.allclose(mine.numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        rows = torch.from_numpy(np.ascontiguousarray(oracle.project(part, X)))
        got = [torch.zeros_like(rows) for _ in range(world)]
        dist.all_gather(got, rows)
        assert np.allclose(torch.cat(got).numpy(), oracle.project(full, X), rtol=1e-12, atol=1e-14)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_slices_and_views():
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    mp.spawn(_worker, args=(2, _free_port()), nprocs=2, join=True)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    """Under torchrun the oracle arm is timed by rank 0 alone; other ranks exit
    without work or output."""
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 0
    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""
