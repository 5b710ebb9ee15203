"""Walker sharding across GPUs (one process per GPU).

Walkers are independent and a walker's trajectory depends only on (seed,
global walker id, step), so a population is split into contiguous ranges of
global ids, one per rank, with no exchange during the walk (weak scaling:
every rank runs its own walkers).  The collectives, all outside the walk: the
collection of the best scheme (an all-reduce-min over (best rank, global
walker id) packed into one int64, then a broadcast of the winning scheme from
its owner), the sums of counters and rank histograms, and, in the exploratory
search, the per-format best schemes that every rank's Resize moves start from.
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


def allreduce_counts(values, device=None) -> np.ndarray:
    """Element-wise sum over ranks of an int64 vector (walker counters, rank
    histograms); every rank receives the sums."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(values, dtype=np.int64), device=device).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def sync_bests(local: dict, term_lens: dict, max_terms: dict, device=None) -> dict:
    """Population synchronisation of the exploratory search across ranks: for
    every format (the same keys, iterated in sorted order, on every rank) the
    global best scheme from each rank's (rank of scheme, global walker id,
    scheme).  Returns {format: (rank of scheme, walker id, scheme)}."""
    out = {}
    for f in sorted(local):
        r, w, sch = local[f]
        out[f] = collect_best_across_ranks(r, w, sch, max_terms=max_terms[f], term_len=term_lens[f], device=device)
    return out
