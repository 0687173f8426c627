"""The benchmark's multi-GPU form splits one search over the ranks: each covers
a shard of the exact screen, and the shards' best pairs are gathered and
merged.  Its host logic runs here as two gloo ranks on the CPU: the gather of
variable-length lists, the merge, and the whole-job timing (the slowest rank)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench

    wl = bench._workload("ising_n2000_m1000", "cpu", N=60, M=40, sweeps=5)
    t, u = bench._reduce_over_ranks(1.0 + rank, 10.0 * (rank + 1), "cpu")
    np.save(os.path.join(out, f"r{rank}.npy"), wl.X)
    with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
        f.write(f"{wl.N} {wl.M} {wl.lam!r} {t!r} {u!r}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_same_data_and_reduction(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [open(tmp_path / f"r{k}.txt").read().split() for k in range(world)]
    X = [np.load(tmp_path / f"r{k}.npy") for k in range(world)]
    # a split search: every rank generates the same data
    assert r[0][:3] == r[1][:3]
    assert np.array_equal(X[0], X[1])
    # whole-job figures on every rank: the slowest time (and the units of all ranks)
    for k in range(world):
        assert float(r[k][3]) == 2.0 and float(r[k][4]) == 30.0


def test_single_process_reduction_is_the_identity():
    import bench

    assert bench._reduce_over_ranks(1.5, 7.0, "cpu") == (1.5, 7.0)


def _shard_main(rank, world, port, out):
    """One rank of a split best-pairs search on the CPU: the shard's m best come
    from the FP64 oracle over the rank's share of the pairs (a stand-in for the
    GPU screen's shard), the gather is the module's, and the selection of the m
    best of the union stands in for recon_select_best."""
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    from oracle import oracle
    from paper_2401_01404_gb300 import inputs, shards

    wl = inputs.config("ising_n100_m200", N=40, M=120, sweeps=30)
    o = oracle.IsingOracle(wl.X, inputs.default_lambda(wl.N, wl.M, 0.5))
    allp = oracle.all_pairs(np.arange(wl.N))
    g, _ = o.score(allp)
    kappa = 1.5
    m = shards.best_m(wl.N, kappa)

    def ordered(p, d):
        o_ = np.lexsort((p[:, 1], p[:, 0], d))
        return p[o_], d[o_]

    def shard_best(ctx, k, kappa_, N):
        mine = (allp[:, 0] * 7 + allp[:, 1]) % world == rank  # this rank's share of the pairs
        p, d = ordered(allp[mine], (-g[mine]).astype(np.float32))
        return p[:m], d[:m]

    def select(P, D, m_):
        key = P[:, 0].astype(np.int64) * wl.N + P[:, 1]
        _, first = np.unique(key, return_index=True)
        p, d = ordered(P[first], D[first])
        return p[:m_], d[:m_]

    assert shards.shard_options(rank, world) == {"shard_index": rank, "shard_count": world}
    p, d = shards.best_pairs_sharded(None, 4, kappa, wl.N, select=select, best_pairs=shard_best)
    np.save(os.path.join(out, f"s{rank}_p.npy"), p)
    np.save(os.path.join(out, f"s{rank}_d.npy"), d)
    if rank == 0:
        pe, de = ordered(allp, (-g).astype(np.float32))
        np.save(os.path.join(out, "ex_p.npy"), pe[:m])
        np.save(os.path.join(out, "ex_d.npy"), de[:m])
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_search_equals_the_whole(tmp_path):
    """Every rank ends with the m best pairs of all pairs: the union of the
    shards' m best holds the global m best, and one gather of variable-length
    lists brings them together."""
    world = 2
    mp.spawn(_shard_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    pe, de = np.load(tmp_path / "ex_p.npy"), np.load(tmp_path / "ex_d.npy")
    for r in range(world):
        p, d = np.load(tmp_path / f"s{r}_p.npy"), np.load(tmp_path / f"s{r}_d.npy")
        assert np.array_equal(p, pe) and np.array_equal(d, de)


def test_shard_options_of_one_process():
    from paper_2401_01404_gb300 import shards

    assert shards.shard_options(0, 1) == {}
    with pytest.raises(ValueError):
        shards.shard_options(2, 2)
    assert shards.best_m(10, 100.0) == 45 and shards.best_m(1000, 1.0) == 1000
