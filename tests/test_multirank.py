"""The benchmark's multi-GPU form is independent replicas, one per rank, with
the whole-job figures reduced over the ranks (slowest time, all units).  Its
host logic runs here as two gloo ranks on the CPU."""
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

    wl = bench._workload("ising_n2000_m1000", rank, "cpu", N=60, M=40, sweeps=5)
    t, u = bench._reduce_over_ranks(1.0 + rank, 10.0 * (rank + 1), "cpu")
    np.save(os.path.join(out, f"r{rank}.npy"), wl.X)
    with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
        f.write(f"{wl.N} {wl.M} {wl.lam!r} {t!r} {u!r}")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_replicas_and_reduction(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r = [open(tmp_path / f"r{k}.txt").read().split() for k in range(world)]
    X = [np.load(tmp_path / f"r{k}.npy") for k in range(world)]
    # replicas: same sizes and penalty, independent samples
    assert r[0][:3] == r[1][:3]
    assert X[0].shape == X[1].shape and not np.array_equal(X[0], X[1])
    # whole-job figures on every rank: the slowest time, the units of all ranks
    for k in range(world):
        assert float(r[k][3]) == 2.0 and float(r[k][4]) == 30.0


def test_single_process_reduction_is_the_identity():
    import bench

    assert bench._reduce_over_ranks(1.5, 7.0, "cpu") == (1.5, 7.0)
