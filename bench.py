#!/usr/bin/env python3
"""Benchmark of the flip-graph walkers on GB300.

Workload (default): the (3,3,3) populations from the naive rank-27 scheme,
Z_T and Z_2, 65536 walkers each, plateau 5e4, uniform proposal.  One bench
step = every walker advances `--chunk` steps (default 50,000; 20 bench steps
make the full 1e6-step budget), then every walker's best scheme is checked
against Eq. (1) on the device and the best scheme of each population is
collected, re-verified on the host and copied out.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "verified flips/sec and reductions per 1e9 flips at 1 GB300, learned vs uniform proposal"
KERNEL_SRCS = [os.path.join(ROOT, "paper_2511_20317_gb300", "csrc", f)
               for f in ("walk_solo.cuh", "walk_group.cuh", "pterm.cuh", "walk_solo_zt32.cu", "walk_solo_z232.cu")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "walk_kernel_333_dram_traffic.txt")

# Algorithmic integer work per walker-step (word operations on 32-bit words):
# candidate search 8 word tests per other slot in Z_T (u, v exact: 2 words each;
# w exact or negated: 4), 3 in Z_2; the two new factors of a flip 2 x 9
# (validity 3 + result 6) in Z_T, 2 XOR in Z_2; the reduction check of an
# accepted flip re-tests both modified terms against every other slot; one
# Philox4x32-10 draw of 10 rounds x 10 integer operations.
C_SEARCH = {0: 8, 1: 3}
C_FLIP = {0: 18, 1: 2}
C_PHILOX = 100


def algorithmic_ops(mode, steps, accepted, rejected, mean_r, word_mult=1, philox=True):
    cs = C_SEARCH[mode] * (mean_r - 1)
    return word_mult * (steps * (cs + (C_PHILOX if philox else 0)) + (accepted + rejected) * C_FLIP[mode] +
                        accepted * 2 * cs)


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SRCS:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def recorded_traffic():
    """DRAM bytes of one bench step's walk-kernel launches from the committed ncu
    summary, when it was taken on the current kernel sources (else None)."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_sha256_16") != kernel_hash():
            return None
        return float(kv["dram_bytes_per_step_walk_launches"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def populations(args):
    from paper_2511_20317_gb300 import workloads as wl
    if args.workload == "333":
        return [((3, 3, 3), 0, wl.naive_start(3, 3, 3), args.walkers),
                ((3, 3, 3), 1, wl.naive_start(3, 3, 3), args.walkers)], 50_000
    if args.workload == "222":
        return [((2, 2, 2), 0, wl.naive_start(2, 2, 2), 1024)], 10_000
    if args.workload == "large":
        from paper_2511_20317_gb300 import starts
        return starts.large_populations(args.walkers), 50_000
    if args.workload == "mixed":
        w = wl.workload_mixed()
        return [(p.fmt, 0, p.start_scheme(), p.walkers) for p in w.populations], 50_000
    raise SystemExit(f"unknown workload {args.workload}")


DATA = {
    "333": "synthetic: naive rank-27 starts (catalogue starts unavailable)",
    "222": "synthetic: naive rank-8 start",
    "mixed": "synthetic: naive rank-mnp starts",
    "large": "synthetic: meta-operator starts built on the host from Strassen's scheme and naive schemes",
}


def workload_name(args, pops, plateau):
    fmts = " + ".join(f"{f[0]}x{f[1]}x{f[2]}{'' if m == 0 else ' Z_2'} r{len(s)} x{n}" for f, m, s, n in pops)
    budget = {"333": "1e6", "222": "1e5", "mixed": "1e6", "large": "1e7"}[args.workload]
    return (f"{args.workload}: {fmts}; {args.chunk} steps per walker per bench step "
            f"({budget} = full budget), plateau {plateau}")


def mapping_name(pop):
    if pop["slots_per_lane"] == 0:
        return "warp per walker, shared-memory signature search"
    if pop["lanes"] == 1:
        sliced = ", bit-sliced slot search" if pop.get("slice_len") else ""
        sliced += " (square factors compiled in)" if pop.get("square") else ""
        return f"thread per walker, {pop['slots_per_lane']} slots{sliced}, {pop['block_threads']} walkers per block"
    return f"{pop['lanes']} lanes x {pop['slots_per_lane']} slots, {pop['block_threads']} threads per block"


def dist_setup(args):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def run_ours(args):
    import torch

    from paper_2511_20317_gb300 import tfg
    rank, world, local = dist_setup(args)
    torch.cuda.set_device(local)
    pops, plateau = populations(args)
    per_rank = sum(p[3] for p in pops)
    params = tfg.tfg_default_params(plateau_len=plateau, walker_id_base=rank * per_rank)
    if args.mapping:
        params.mapping = args.mapping
    params.use_graph = args.graph
    W = tfg.Walkers(pops, seed=args.seed, params=params)
    lanes = W.autotune(trial_steps=300, trial_walkers=65536) if args.autotune else None
    stream = W.stream
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")   # > 129 MB L2
    fails = torch.zeros(1, dtype=torch.int64, device="cuda")
    L = tfg.lib()
    import ctypes

    def step():
        W.walk(args.chunk)
        tfg._check(L.tfg_verify_all_async(W.ctx, ctypes.c_void_p(fails.data_ptr())))

    def collect():
        out = []
        for f in range(W.n_formats):
            out.append(W.collect_best(f)[1])
        return out

    for _ in range(args.warmup):
        step()
        collect()
    st0, _ = W.stats()
    st0_f = [W.stats(f)[0] for f in range(W.n_formats)]
    W.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    t_wall = time.perf_counter()
    verify_failures = 0
    best_ranks = None
    for k in range(args.steps):
        flush.zero_()                                # L2 flush between timed steps (untimed)
        with torch.cuda.stream(stream):
            ev[k][0].record(stream)
            W.walk(args.chunk)
            ev[k][1].record(stream)
            tfg._check(L.tfg_verify_all_async(W.ctx, ctypes.c_void_p(fails.data_ptr())))
        best_ranks = collect()                       # argmin + device and host verification + D2H
        with torch.cuda.stream(stream):
            ev[k][2].record(stream)
        verify_failures += int(fails.item())
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(args.steps)]
    walk_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    t_total = sum(step_ms) / 1e3
    st1, hist = W.stats()
    walker_steps = st1["steps"] - st0["steps"]
    assert walker_steps == per_rank * args.chunk * args.steps
    # max over ranks
    t_max = t_total
    if world > 1:
        tt = torch.tensor([t_total], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    total_steps = walker_steps * world
    # the metric counts applied flips: steps whose flip passed the ternary check and was made
    applied = sum(W.stats(f)[0]["accepted"] - st0_f[f]["accepted"] for f in range(W.n_formats))
    if world > 1:
        ta = torch.tensor([applied], dtype=torch.int64, device="cuda")
        torch.distributed.all_reduce(ta)
        applied = int(ta.item())
    value = applied / t_max
    steps_per_s = total_steps / t_max

    # roofline of the walk kernel: algorithmic integer ops per launch / launch time
    ops, ops_nophilox = 0.0, 0.0
    per_mode = {}
    for f, (fmt, mode, _, nw) in enumerate(pops):
        a0, a1 = st0_f[f], W.stats(f)[0]
        info, _, _ = W.read_walkers(W.pop[f]["first"], min(nw, 4096), slots=False, best=False)
        mean_r = float(info["r"].mean())
        steps_f = a1["steps"] - a0["steps"]
        acc, rej = a1["accepted"] - a0["accepted"], a1["rejected"] - a0["rejected"]
        ops += algorithmic_ops(mode, steps_f, acc, rej, mean_r)
        ops_nophilox += algorithmic_ops(mode, steps_f, acc, rej, mean_r, philox=False)
        per_mode[f"{'ZT' if mode == 0 else 'Z2'} {fmt[0]}x{fmt[1]}x{fmt[2]}"] = {
            "lowest_rank": a1["min_best_r"], "mean_live_rank": round(mean_r, 2),
            "rank_hist": {int(k): int(v) for k, v in enumerate(W.stats(f)[1]) if v},
            "accepted_frac": round(acc / max(steps_f, 1), 4),
            "reductions_per_1e9_flips": round((a1["reductions"] - a0["reductions"]) / max(acc, 1) * 1e9, 1),
            "mapping": mapping_name(W.pop[f])}
    walk_s = sum(walk_ms) / 1e3
    achieved = ops / walk_s / 1e12          # Tops/s
    # integer ALU pipe: one warp instruction per 2 cycles per SM sub-partition (16 lanes/clk),
    # 4 sub-partitions x 152 SMs at the 2070 MHz maximum SM clock
    alu_peak = 152 * 4 * 16 * 2.07e9 / 1e12
    traffic = recorded_traffic() if args.workload == "333" else None   # the capture is of that workload

    # end to end through the public API with host buffers: the walkers' state lives
    # in pinned host memory between steps, as for a caller that keeps it there.
    # Per step: tfg_restore (H2D of the whole state), walk, verify every best
    # scheme, collect each population's best scheme to the host, read the
    # counters, tfg_checkpoint (D2H of the whole state).  The state continues
    # the timed run's trajectories (a context created with the same arguments),
    # so the step covers the same phase of the walk as the timed steps.
    e2e_steps = max(1, min(args.steps, 3))
    import ctypes as _ct
    L_ = tfg.lib()
    used = _ct.c_size_t()
    tfg._check(L_.tfg_checkpoint(W.ctx, None, 0, _ct.byref(used)))
    host_state = torch.empty(used.value, dtype=torch.uint8, pin_memory=True)
    tfg._check(L_.tfg_checkpoint(W.ctx, _ct.c_void_p(host_state.data_ptr()), used.value, _ct.byref(used)))
    E = tfg.Walkers(pops, seed=args.seed, params=params)
    if lanes is not None:
        E.autotune(trial_steps=300, trial_walkers=65536)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h, e2e_applied = 0, 0
    for _ in range(e2e_steps):
        tfg._check(L_.tfg_restore(E.ctx, _ct.c_void_p(host_state.data_ptr()), used.value))
        a0 = E.stats()[0]["accepted"]
        E.walk(args.chunk)
        E.verify_all()
        for f in range(E.n_formats):
            sch, r, w = E.collect_best(f)
            d2h += sch.nbytes + 12
        e2e_applied += E.stats()[0]["accepted"] - a0
        tfg._check(L_.tfg_checkpoint(E.ctx, _ct.c_void_p(host_state.data_ptr()), used.value, _ct.byref(used)))
        d2h += used.value + 2 * 8 * 11
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    h2d = used.value
    E.close()
    e2e_val = e2e_applied * world / e2e_t

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "flips/s",
        "walker_steps_per_s": steps_per_s,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": DATA[args.workload],
        "config": {"workload": workload_name(args, pops, plateau),
                   "walkers_per_gpu": per_rank, "steps_per_walker_per_step": args.chunk,
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"walker shards x{world}"},
        "modes": per_mode,
        "verified": {"device_checked_best_schemes": per_rank * args.steps, "failures": verify_failures,
                     "collected_best_ranks": best_ranks},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                     "frac": achieved / alu_peak, "traffic": traffic,
                     "frac_excluding_philox": ops_nophilox / walk_s / 1e12 / alu_peak,
                     "kernel": "walk kernels of the step (" + "; ".join(p["mapping"] for p in per_mode.values()) + ")",
                     "walk_ms_per_step": sum(walk_ms) / len(walk_ms)},
        "e2e": {"value": e2e_val, "unit": "flips/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h // e2e_steps},
        "gpu_launches": (2 * W.n_formats + 2 * W.n_formats) * args.steps,
        "clocks": clk,
        "wall_s": wall,
    }
    if lanes is not None:
        line["config"]["autotuned_lanes_per_walker"] = lanes
    if world > 1:
        # the collectives of the sharded path (after the timed region): global best scheme
        # per population, and rank histograms summed over ranks
        from paper_2511_20317_gb300 import shard
        gbest = []
        for f in range(W.n_formats):
            sch, r_, wid = W.collect_best(f)
            g = shard.collect_best_across_ranks(r_, rank * per_rank + wid, sch, W.pop[f]["r_max"], sch.shape[1],
                                                device="cuda")
            gbest.append({"rank": g[0], "walker": g[1]})
        line["global_best"] = gbest
        for f, key in enumerate(per_mode):
            hist = shard.allreduce_counts(W.stats(f)[1], device="cuda")
            per_mode[key]["rank_hist"] = {int(k): int(v) for k, v in enumerate(hist) if v}
            per_mode[key]["lowest_rank"] = gbest[f]["rank"]
    if rank == 0 and args.learned:
        line["learned_vs_uniform"] = learned_ab(args)
    if rank == 0 and args.cpu_baseline:
        cb = oracle_sample(args, pops, plateau)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        # the roofline's op count (counters and the live rank at the end) against the
        # oracle's exact per-step count, on the oracle's sample of the same walkers
        ratio = cb["ops_estimate"] / max(cb["ops_exact"], 1.0)
        line["roofline"]["ops_estimate_over_oracle_count"] = ratio
        line["roofline"]["frac_at_oracle_count"] = line["roofline"]["frac"] / ratio
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def learned_ab(args):
    """The learned proposal against uniform choice over the same candidate
    windows (the learned-proposal workload: (4,4,4) and (3,4,5), 262144 walkers,
    equal step budgets): the network is trained on the device from the
    logged window-uniform walks of the uniform workloads' formats (4096
    walkers x --ab-collect-steps steps each, seeds 100..; label 1 on the
    chosen candidates of the --ab-horizon steps up to each rank-lowering step),
    then both arms run from the naive (4,4,4) and (3,4,5) schemes with 262144
    walkers, plateau 5e4, evaluation seeds 1000..1004: the learned arm for
    --ab-steps steps per walker, the uniform arm for as many steps (equal
    budget) and for the learned arm's wall time (equal time)."""
    from paper_2511_20317_gb300 import learned
    t0 = time.perf_counter()
    entries = learned.collect(walkers=4096, steps=args.ab_collect_steps, horizon=args.ab_horizon)
    params, info = learned.train(entries, epochs=30)
    res = learned.ab_test(params, seeds=tuple(range(args.ab_seeds)), walkers=args.ab_walkers, steps=args.ab_steps)
    return {"workload": f"naive (4,4,4) and (3,4,5), Z_T, {args.ab_walkers} walkers, {args.ab_steps} window steps "
                        f"per walker (learned, and uniform at equal steps) and uniform at the learned arm's wall "
                        f"time; plateau 5e4; {args.ab_seeds} evaluation seeds; eps 0.05; 256-candidate windows",
            "training": {"label_horizon_steps": args.ab_horizon, "collect_steps": args.ab_collect_steps,
                         "samples": info["samples"],
                         "positives": info["positives"],
                         "loss_first": info["loss"][0], "loss_last": info["loss"][-1]},
            "results": res, "seconds": time.perf_counter() - t0}


def oracle_sample(args, pops, plateau):
    """The oracle as it stands, on the host cores, on a bounded sample of the
    bench workload: walkers 0, 256, 512, ... of each population (256 per
    population at the default size), advanced exactly like the GPU walkers --
    warmup + steps chunks of --cpu-chunk steps each (default: the bench's own
    chunk), the timed chunks after the warm-up ones.  Returns the applied
    flips per second of the timed chunks and the per-chunk times.  Both the GPU
    arm's cpu_baseline and the reference arm run this same sample."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    chunk = args.cpu_chunk or args.chunk
    walkers = []
    for fmt, mode, start, nw in pops:
        ids = np.arange(0, nw, max(1, nw // args.cpu_walkers))[:args.cpu_walkers]
        walkers.append(oracle.Walkers(fmt, start, ids, seed=args.seed, mode=mode, plateau_len=plateau))
    n_w = sum(w.walker_ids.size for w in walkers)
    per_step, applied, steps_done = [], 0, 0
    for k in range(args.warmup + args.steps):
        if k == args.warmup:   # counters at the start of the timed chunks
            c0 = [{f: int(w.info[f].astype(np.int64).sum()) for f in ("ops", "t", "accepted", "rejected")}
                  for w in walkers]
        acc0 = sum(int(w.info["accepted"].sum()) for w in walkers)
        t0 = time.perf_counter()
        for w in walkers:
            w.walk(chunk, threads)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            per_step.append(dt)
            applied += sum(int(w.info["accepted"].sum()) for w in walkers) - acc0
            steps_done += n_w * chunk
    t = sum(per_step)
    # the oracle's exact algorithmic op count of the timed chunks, and the estimate the
    # GPU arm's roofline makes from the same kind of inputs (counters, the live rank
    # at the end) for the same walkers
    exact = estimate = 0.0
    for w, c, (fmt, mode, _, _) in zip(walkers, c0, pops):
        exact += float(w.info["ops"].astype(np.int64).sum() - c["ops"])
        estimate += algorithmic_ops(mode, float(w.info["t"].astype(np.int64).sum() - c["t"]),
                                    float(w.info["accepted"].sum() - c["accepted"]),
                                    float(w.info["rejected"].sum() - c["rejected"]), float(w.info["r"].mean()))
    return {"value": applied / t, "unit": "flips/s", "cores": threads, "kind": "oracle",
            "ops_exact": exact, "ops_estimate": estimate,
            "sample": f"{n_w} walkers ({args.cpu_walkers} per population, ids spread over it) advanced "
                      f"{args.warmup} + {args.steps} chunks of {chunk} steps like the GPU walkers; "
                      f"{applied} applied flips in {steps_done} walker-steps over {t:.1f} s timed",
            "ms_per_step": t / max(1, len(per_step)) * 1e3, "walker_steps_per_s": steps_done / t}


def run_reference(args):
    rank, world, _ = dist_setup(args)
    if rank != 0:
        return
    pops, plateau = populations(args)
    cb = oracle_sample(args, pops, plateau)
    value = cb["value"]
    step_walker_steps = sum(p[3] for p in pops) * args.chunk
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "flips/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["ms_per_step"],
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i8", "data": "synthetic",
            "config": {"workload": "333: 3x3x3 naive27 Z_T + Z_2, the oracle on a bounded sample of the "
                                   "walkers on the host cores",
                       "sample_walkers": args.cpu_walkers * len(pops),
                       "steps_per_walker_per_step": args.cpu_chunk or args.chunk},
            "walker_steps_per_s": cb["walker_steps_per_s"],
            "full_step_extrapolated_ms": step_walker_steps / cb["walker_steps_per_s"] * 1e3,
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": value, "unit": "flips/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="333")
    ap.add_argument("--walkers", type=int, default=65536)
    ap.add_argument("--chunk", type=int, default=50_000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--mapping", type=int, default=0)
    ap.add_argument("--graph", type=int, default=2, help="0 plain launches, 1 chained graph, 2 forked graph (default: the two populations run concurrently)")
    ap.add_argument("--cpu-walkers", type=int, default=256, help="oracle sample: walkers per population")
    ap.add_argument("--cpu-chunk", type=int, default=0, help="oracle sample: steps per chunk (0: --chunk)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-learned", dest="learned", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--ab-walkers", type=int, default=262144)
    ap.add_argument("--ab-steps", type=int, default=1500)
    ap.add_argument("--ab-seeds", type=int, default=5)
    ap.add_argument("--ab-horizon", type=int, default=16, help="label-1 horizon of the training log (steps)")
    ap.add_argument("--ab-collect-steps", type=int, default=16000, help="window steps of the logged training walks")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        spawn_ranks(args.gpus)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


def spawn_ranks(n: int):
    """--gpus N without an outside launcher: re-run this script as N ranks on
    this node under torch.distributed.run (one process per GPU, rendezvous on
    127.0.0.1) and exit with its status."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    sys.exit(subprocess.call(cmd))


if __name__ == "__main__":
    main()
