"""Walker sharding across GPUs (one process per GPU).

Walkers are independent and a walker's trajectory depends only on (seed,
global walker id, step), so a population is split into contiguous ranges of
global ids, one per rank, with no exchange during the walk (weak scaling:
every rank runs its own walkers).  The only collective is the collection of
the best scheme: an all-reduce-min over (best rank, global walker id) packed
into one int64, then a broadcast of the winning scheme from its owner.
"""
from __future__ import annotations

import numpy as np


def shard_range(rank: int, world: int, total: int) -> tuple[int, int]:
    """[first, first + count) of `total` walkers for `rank` of `world`: the
    remainder goes to the lowest ranks, so the ranges tile [0, total)."""
    base, extra = divmod(total, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def pack_best(rank_of_scheme: int, walker_id: int) -> int:
    return (int(rank_of_scheme) << 40) | int(walker_id)


def unpack_best(key: int) -> tuple[int, int]:
    return key >> 40, key & ((1 << 40) - 1)


def collect_best_across_ranks(local_rank_of_scheme: int, local_walker_id: int, local_scheme: np.ndarray,
                              max_terms: int, term_len: int, device=None):
    """Global best scheme over all ranks (ties: lowest global walker id).
    Returns (rank_of_scheme, walker_id, scheme int8 [r, term_len]) on every rank."""
    import torch
    import torch.distributed as dist
    key = torch.tensor([pack_best(local_rank_of_scheme, local_walker_id)], dtype=torch.int64, device=device)
    dist.all_reduce(key, op=dist.ReduceOp.MIN)
    best_rank, best_walker = unpack_best(int(key.item()))
    mine = (best_rank == local_rank_of_scheme and best_walker == local_walker_id)
    owner = torch.tensor([dist.get_rank() if mine else dist.get_world_size()], dtype=torch.int64, device=device)
    dist.all_reduce(owner, op=dist.ReduceOp.MIN)
    buf = torch.zeros(max_terms * term_len, dtype=torch.int8, device=device)
    if mine:
        flat = torch.from_numpy(np.ascontiguousarray(local_scheme, dtype=np.int8).reshape(-1))
        buf[: flat.numel()] = flat.to(buf.device)
    dist.broadcast(buf, src=int(owner.item()))
    scheme = buf.cpu().numpy()[: best_rank * term_len].reshape(best_rank, term_len)
    return best_rank, best_walker, scheme
