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


def _pdd_rank_main(rank, world, port, out_dir):
    """Rank r solves its shard of the nodal points, all-gathers the nodal values (the method's one
    exchange), then solves its own range of the decoupled subdomains; the CPU oracle stands in for
    both GPU stages."""
    import torch
    import torch.distributed as dist

    import oracle
    from oracle import pdd
    from paper_2402_06491_gb300.sharding import pdd_subdomain_range

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pb = dict(workloads.problem_pdd_3d(), D=0.3)
    grid = dict(dim=2, lo=[0.0, 0.0], hi=[3.0, 2.0], sub=[3, 2], cells=[6, 6], nodes=[5, 5], t_nodes=3, T=0.3,
                nsteps=6)
    pb2 = dict(pb, dim=2, u0=("tanh_prod", (0.0, 1.0, 1.5, 1.0)))
    x, t = pdd.points(grid)
    n = x.shape[0]
    a, b = shard_range(n, world, rank)
    r = oracle.solve(pb2, x[a:b], t[a:b], np.full(b - a, 300, np.uint64), 6, 3, 3, 0, point_base=a, nthreads=1)
    counts = [shard_range(n, world, k)[1] - shard_range(n, world, k)[0] for k in range(world)]
    mine = torch.zeros(max(counts), dtype=torch.float64)
    mine[: b - a] = torch.from_numpy(r["u"])
    parts = [torch.zeros(max(counts), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, mine)
    u_nodes = np.concatenate([parts[k][: counts[k]].numpy() for k in range(world)])
    s0, s1 = pdd_subdomain_range(grid, world, rank)
    part = pdd.pdd_solve(pb2, grid, u_nodes, subdomains=(s0, s1))
    np.save(os.path.join(out_dir, f"pdd_{rank}.npy"), part)
    np.save(os.path.join(out_dir, f"nodes_{rank}.npy"), u_nodes)
    dist.destroy_process_group()


def test_pdd_subdomains_shard_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    from oracle import pdd

    world, port = 2, 29000 + (os.getpid() % 2000)
    mp.start_processes(_pdd_rank_main, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn")
    nodes = [np.load(os.path.join(tmp_path, f"nodes_{k}.npy")) for k in range(world)]
    assert np.array_equal(nodes[0], nodes[1])
    parts = [np.load(os.path.join(tmp_path, f"pdd_{k}.npy")) for k in range(world)]
    pb2 = dict(workloads.problem_pdd_3d(), D=0.3, dim=2, u0=("tanh_prod", (0.0, 1.0, 1.5, 1.0)))
    grid = dict(dim=2, lo=[0.0, 0.0], hi=[3.0, 2.0], sub=[3, 2], cells=[6, 6], nodes=[5, 5], t_nodes=3, T=0.3,
                nsteps=6)
    full = pdd.pdd_solve(pb2, grid, nodes[0])
    # interiors are disjoint (zero elsewhere) and plane nodes identical: rank 0's planes + both interiors
    planes = np.zeros(full.shape, bool)
    planes[::6, :] = True
    planes[:, ::6] = True
    combined = np.where(planes, parts[0], parts[0] + parts[1])
    assert np.array_equal(combined, full)


BATCH = 1500


def _fault_rank_main(rank, world, port, out_dir):
    """Trees of each point cut into batches of BATCH, batch b on rank b % world; rank 1 loses its batch 1
    (an exception on the host: the batch's sums never reach the exchange).  Every rank sends, per point
    and batch, the order sums of its completed batches and the trees they hold; the dropped batch
    contributes nothing, and the trees it would have held are not counted."""
    import torch
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = workloads.subsample(workloads.workload_sin_2d(), 3, ntrees=6000)
    K, n = wl["K"], wl["x"].shape[0]
    nb = (6000 + BATCH - 1) // BATCH
    sums = torch.zeros((n, nb, K + 3), dtype=torch.float64)  # S1 per kept order, pruned count, trees
    for p in range(n):
        for b in range(rank, nb, world):
            rec = oracle.trees(wl["problem"], wl["x"][p], float(wl["t"][p]), p, b * BATCH, BATCH, K, wl["seed"])
            try:
                if rank == 1 and b == 1:
                    np.save(os.path.join(out_dir, f"lost_{p}.npy"), rec["w"])  # what the rank had computed
                    raise RuntimeError("rank 1 lost batch 1")
                for o in range(K + 1):
                    sums[p, b, o] = float(np.sum(rec["w"][rec["order"] == o]))
                sums[p, b, K + 1] = float(np.sum(rec["order"] > K))
                sums[p, b, K + 2] = BATCH
            except RuntimeError:
                pass
    dist.all_reduce(sums)
    if rank == 0:
        np.save(os.path.join(out_dir, "sums.npy"), sums.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_dropped_tree_batches_leave_an_estimate_over_the_trees_done(tmp_path):
    """Fault tolerance from independent samples (Sec. 3): when a rank loses a batch of trees, the
    combined a_n = S1_n / N_done is the estimate over exactly the trees that were walked (checked
    against the oracle's records of those trees), and the lost batch re-run on another rank gives the
    same tree weights bit for bit (the streams are keyed by point, tree and node label)."""
    pytest.importorskip("torch")
    import socket

    import torch.multiprocessing as mp

    import oracle

    oracle.build()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_fault_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    sums = np.load(tmp_path / "sums.npy")
    wl = workloads.subsample(workloads.workload_sin_2d(), 3, ntrees=6000)
    K = wl["K"]
    for p in range(sums.shape[0]):
        n_done = sums[p, :, K + 2].sum()
        assert n_done == 6000 - BATCH
        a = sums[p, :, :K + 1].sum(axis=0) / n_done
        kept = [b for b in range(sums.shape[1]) if b != 1]
        rec = [oracle.trees(wl["problem"], wl["x"][p], float(wl["t"][p]), p, b * BATCH, BATCH, K, wl["seed"])
               for b in kept]
        w = np.concatenate([r["w"] for r in rec])
        order = np.concatenate([r["order"] for r in rec])
        expect = np.array([w[order == o].sum() for o in range(K + 1)]) / n_done
        assert np.allclose(a, expect, rtol=1e-13, atol=1e-15)
        again = oracle.trees(wl["problem"], wl["x"][p], float(wl["t"][p]), p, BATCH, BATCH, K, wl["seed"])
        assert np.array_equal(again["w"], np.load(tmp_path / f"lost_{p}.npy"))
