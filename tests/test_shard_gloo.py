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


def _rank_sync(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local, lens, caps = {}, {}, {}
    counts = []
    for fmt in [(2, 2, 2), (2, 2, 3)]:
        first, count = shard.shard_range(rank, world, TOTAL)
        W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(first, first + count), seed=SEED,
                           plateau_len=L).walk(STEPS, threads=1)
        w = int(np.lexsort((np.arange(count), W.info["best_r"]))[0])
        local[fmt] = (int(W.info["best_r"][w]), first + w, W.best_scheme(w))
        lens[fmt], caps[fmt] = W.LT, W.r_max
        hist = np.bincount(W.info["best_r"], minlength=40)
        counts.append(np.concatenate([[W.info["accepted"].sum(), W.info["merges"].sum()], hist]))
    got = shard.sync_bests(local, lens, caps)
    sums = shard.allreduce_counts(np.concatenate(counts))
    np.save(os.path.join(out_dir, f"sums{rank}.npy"), sums)
    for fmt, (r, w, sch) in got.items():
        np.save(os.path.join(out_dir, f"sync{rank}_{fmt[2]}.npy"), np.concatenate([[r, w], sch.reshape(-1)]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_population_sync_and_counter_sums(tmp_path):
    """The exploratory search's population synchronisation across ranks gives every
    rank the per-format global best (lowest rank, then walker id); counters and
    rank histograms sum to the whole population's."""
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_sync, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    want_counts = []
    for fmt in [(2, 2, 2), (2, 2, 3)]:
        whole = oracle.Walkers(fmt, naive_start(*fmt), np.arange(TOTAL), seed=SEED, plateau_len=L).walk(STEPS)
        hist = np.bincount(whole.info["best_r"], minlength=40)
        want_counts.append(np.concatenate([[whole.info["accepted"].sum(), whole.info["merges"].sum()], hist]))
        order = np.lexsort((np.arange(TOTAL), whole.info["best_r"]))
        br, bw = int(whole.info["best_r"][order[0]]), int(order[0])
        for r in range(world):
            got = np.load(tmp_path / f"sync{r}_{fmt[2]}.npy")
            assert (int(got[0]), int(got[1])) == (br, bw)
            assert np.array_equal(got[2:].reshape(br, -1), whole.best_scheme(bw))
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"sums{r}.npy"), np.concatenate(want_counts))


def test_bench_spawns_its_own_ranks_for_gpus_2():
    """bench.py --gpus 2 without an outside launcher starts two ranks itself
    (torch.distributed.run on 127.0.0.1); the reference arm runs on rank 0 and
    prints one JSON line with n_gpus = 2, the other rank exits 0.  CPU only:
    the reference arm uses gloo and no GPU."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "1", "--cpu-walkers", "2", "--cpu-chunk", "300"],
                         capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["ms_per_step"] > 0 and rec["e2e"]["value"] == rec["value"]
