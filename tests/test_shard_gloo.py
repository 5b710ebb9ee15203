"""Multi-rank walker sharding on CPU (gloo, world size 2): the ranges tile the
population, the sharded walk equals one whole walk, and the best-scheme
collective picks the global minimum (ties to the lowest walker id).  The walk
itself is the oracle's here (no GPU); on GPUs each rank runs libtfg with
tfg_params.walker_id_base = its first id."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2511_20317_gb300 import shard
from paper_2511_20317_gb300.workloads import naive_start


def test_shard_ranges_tile_the_population():
    for total in [0, 1, 7, 1024, 65537]:
        for world in [1, 2, 3, 8]:
            ranges = [shard.shard_range(r, world, total) for r in range(world)]
            assert sum(c for _, c in ranges) == total
            pos = 0
            for first, count in ranges:
                assert first == pos
                pos += count
            assert max(c for _, c in ranges) - min(c for _, c in ranges) <= 1


def test_pack_order_is_rank_then_walker():
    keys = [shard.pack_best(r, w) for r, w in [(7, 5), (7, 3), (6, 900), (8, 0)]]
    assert min(keys) == shard.pack_best(6, 900)
    assert shard.unpack_best(shard.pack_best(23, 123456)) == (23, 123456)
    assert min(shard.pack_best(7, 5), shard.pack_best(7, 3)) == shard.pack_best(7, 3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


FMT, TOTAL, STEPS, SEED, L = (2, 2, 2), 40, 3000, 13, 300


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = shard.shard_range(rank, world, TOTAL)
    W = oracle.Walkers(FMT, naive_start(*FMT), np.arange(first, first + count), seed=SEED,
                       plateau_len=L).walk(STEPS, threads=1)
    np.save(os.path.join(out_dir, f"info{rank}.npy"), W.info)
    np.save(os.path.join(out_dir, f"slots{rank}.npy"), W.slots)
    w = int(np.lexsort((np.arange(count), W.info["best_r"]))[0])
    best_r, best_w, scheme = shard.collect_best_across_ranks(
        int(W.info["best_r"][w]), first + w, W.best_scheme(w), max_terms=W.r_max, term_len=W.LT)
    np.save(os.path.join(out_dir, f"best{rank}.npy"), np.array([best_r, best_w]))
    np.save(os.path.join(out_dir, f"scheme{rank}.npy"), scheme)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_equal_single_run(tmp_path):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    whole = oracle.Walkers(FMT, naive_start(*FMT), np.arange(TOTAL), seed=SEED, plateau_len=L).walk(STEPS)
    info = np.concatenate([np.load(tmp_path / f"info{r}.npy") for r in range(world)])
    slots = np.concatenate([np.load(tmp_path / f"slots{r}.npy") for r in range(world)])
    assert np.array_equal(info, whole.info) and np.array_equal(slots, whole.slots)
    # the collective's winner: lowest best rank, then lowest walker id, seen by every rank
    order = np.lexsort((np.arange(TOTAL), whole.info["best_r"]))
    want = (int(whole.info["best_r"][order[0]]), int(order[0]))
    for r in range(world):
        got = tuple(int(v) for v in np.load(tmp_path / f"best{r}.npy"))
        assert got == want
        sch = np.load(tmp_path / f"scheme{r}.npy")
        assert np.array_equal(sch, whole.best_scheme(want[1]))
        assert oracle.brent_valid(FMT, sch)
