"""Points shard over ranks with no data-path collective: each rank solves a
contiguous slice with point_base = its first global index, and the slices
reproduce the one-rank solve bit for bit (the counter-based streams are keyed
by the global point index).  Exercised with 2 gloo ranks on the CPU, the
compute done by the oracle."""
import os

import numpy as np
import pytest

import workloads
from paper_2402_06491_gb300.sharding import shard_range


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (7, 2), (16, 3), (512, 8), (5, 8)])
def test_shard_range_partitions(n, world):
    covered = []
    for r in range(world):
        a, b = shard_range(n, world, r)
        assert 0 <= a <= b <= n
        covered.extend(range(a, b))
        assert (b - a) in (n // world, n // world + 1)
    assert covered == list(range(n))


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = workloads.subsample(workloads.workload_sin_2d(), 10, ntrees=1500)
    n = wl["x"].shape[0]
    a, b = shard_range(n, world, rank)
    r = oracle.solve(wl["problem"], wl["x"][a:b], wl["t"][a:b], wl["ntrees"][a:b], wl["K"], wl["L"], wl["M"],
                     wl["seed"], point_base=a, nthreads=1)
    import torch

    u = torch.zeros(n, dtype=torch.float64)
    u[a:b] = torch.from_numpy(r["u"])
    dist.all_reduce(u)  # test harness only: gather the shards to compare them
    if rank == 0:
        np.save(os.path.join(out_dir, "u.npy"), u.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_shards_match_single_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import socket

    import torch.multiprocessing as mp

    import oracle

    oracle.build()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    got = np.load(tmp_path / "u.npy")
    wl = workloads.subsample(workloads.workload_sin_2d(), 10, ntrees=1500)
    full = oracle.solve(wl["problem"], wl["x"], wl["t"], wl["ntrees"], wl["K"], wl["L"], wl["M"], wl["seed"])
    assert np.array_equal(got, full["u"])
