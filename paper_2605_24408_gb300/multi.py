"""Multi-GPU split of the replica space (one process per GPU).

Replicas are independent chains keyed by their global id, so rank r of W
runs global replicas [r R, (r+1) R) with replica_base = r R, and the results
are bit-identical to one process running all W R replicas. The only exchange
is at the end: the smallest best cost over ranks (ties to the lowest global
replica id) and that rank's permutation. Works with any torch.distributed
backend (NCCL on GPUs, gloo on CPU).
"""

from __future__ import annotations

import numpy as np


def shard(rank: int, world: int, replicas_per_rank: int) -> tuple[int, int]:
    """(replica_base, count) of this rank."""
    return rank * replicas_per_rank, replicas_per_rank


def global_best(best_cost: int, best_replica: int, perm, replica_base: int, device=None):
    """Min-reduce (cost, global replica id) over all ranks and broadcast the
    winner's permutation. Returns (cost, global replica id, perm as numpy)."""
    import torch
    import torch.distributed as dist

    dev = device if device is not None else "cpu"
    gid = replica_base + int(best_replica)
    key = torch.tensor([int(best_cost), gid], dtype=torch.int64, device=dev)
    world = dist.get_world_size()
    keys = [torch.zeros_like(key) for _ in range(world)]
    dist.all_gather(keys, key)
    ks = [(int(k[0]), int(k[1]), r) for r, k in enumerate(keys)]
    cost, wid, wrank = min(ks)
    p = torch.as_tensor(np.ascontiguousarray(perm, dtype=np.int32), device=dev)
    dist.broadcast(p, src=wrank)
    return cost, wid, p.cpu().numpy()


def rank_winner(replica_best_cost) -> int:
    """This rank's winning replica (its index within the rank): the smallest
    best cost, ties to the lowest index."""
    c = np.asarray(replica_best_cost, dtype=np.int64)
    return int(np.argmin(c))  # argmin returns the first of equal minima


def rank_result(replica_best_cost, best_perm, replica_base: int, device=None):
    """The final answer of a sharded run from one rank's per-replica best
    costs and its best permutation (the permutation of its winning replica):
    (cost, global replica id, perm) agreed by every rank."""
    w = rank_winner(replica_best_cost)
    return global_best(int(np.asarray(replica_best_cost)[w]), w, best_perm, replica_base, device)
