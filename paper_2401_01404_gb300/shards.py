"""A best-pairs search split over several processes, one GPU each.

The exact screen (recon_options.knn_mode = RECON_KNN_SCREEN) covers every pair
of the upper triangle in 128 x 256 blocks; with shard_count = world a context
covers only every world-th block (shard_index = its rank).  Each rank returns
the m best pairs of its shard: the global m best pairs lie in the union of the
shards' lists, so one all-gather of those lists (the search's only exchange
step) and a selection of the m best of their union (recon_select_best, on the
GPU) give the unsharded answer exactly.  This module holds that host logic:
the shard options of a rank, the gather of variable-length lists over a
torch.distributed group, and the merge.  The scores themselves are computed by
the library; nothing here does any of the method's arithmetic.
"""
from __future__ import annotations

import numpy as np


def shard_options(rank: int, world: int) -> dict:
    """recon_options fields of rank `rank` of `world` (none for a single process)."""
    if world <= 1:
        return {}
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside [0, {world})")
    return {"shard_index": int(rank), "shard_count": int(world)}


def best_m(N: int, kappa: float) -> int:
    """m = round(kappa N) (half up), at most the number of pairs."""
    return min(int(np.floor(kappa * N + 0.5)), N * (N - 1) // 2)


def gather_lists(pairs: np.ndarray, d: np.ndarray, group=None):
    """All-gather of each rank's (pairs [n x 2] int32, d [n] float32), lists of
    different lengths: the lengths first, then the lists padded to the longest.
    Returns the concatenation in rank order.  On an NCCL group the exchange goes
    through the current CUDA device; on gloo through host memory."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    d = np.ascontiguousarray(np.asarray(d, dtype=np.float32).ravel())
    n = torch.tensor([len(d)], dtype=torch.int64, device=dev)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    counts = [int(x.item()) for x in ns]
    top = max(max(counts), 1)
    pp = torch.zeros((top, 2), dtype=torch.int32, device=dev)
    dd = torch.zeros((top,), dtype=torch.float32, device=dev)
    pp[: len(d)] = torch.from_numpy(pairs).to(dev)
    dd[: len(d)] = torch.from_numpy(d).to(dev)
    gp = [torch.empty_like(pp) for _ in range(world)]
    gd = [torch.empty_like(dd) for _ in range(world)]
    dist.all_gather(gp, pp, group=group)
    dist.all_gather(gd, dd, group=group)
    P = np.concatenate([gp[r][: counts[r]].cpu().numpy() for r in range(world)]) if sum(counts) else pairs[:0]
    D = np.concatenate([gd[r][: counts[r]].cpu().numpy() for r in range(world)]) if sum(counts) else d[:0]
    return P, D


def best_pairs_sharded(ctx, k: int, kappa: float, N: int, group=None, select=None, best_pairs=None):
    """The m best pairs of a split search, on every rank of `group`: this rank's
    shard (recon_best_pairs on a context made with shard_options), the gather,
    and the selection of the m best of the union (recon_select_best on ctx).
    `select(pairs, d, m)` and `best_pairs(ctx, k, kappa, N)` replace the library
    calls (tests of the host logic without a GPU)."""
    from . import recon as R

    bp = best_pairs or R.recon_best_pairs
    p, d = bp(ctx, k, kappa, N)
    P, D = gather_lists(p, d, group)
    m = best_m(N, kappa)
    if select is None:
        return R.recon_select_best(ctx, P, D, m)
    return select(P, D, m)
