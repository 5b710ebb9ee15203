"""Search driver: run a walker population to a step budget and report what the
flip-graph walks found.

    python -m paper_2511_20317_gb300.search --workload 333 --steps 1000000
    python -m paper_2511_20317_gb300.search --workload large --steps 100000 --lift-333-steps 200000

Z_2 populations also report the Z_2 -> Z_T sign lifting (the paper's ternary
lifting step) of the best schemes of their lowest-rank walkers.

For every population it prints one JSON line with the lowest rank reached, the
histogram of the walkers' best ranks, the number of walkers at the lowest
rank, and the best scheme's rank, naive additive complexity and isotropy
invariants (type polynomial, rank sums) after an independent host check of
Eq. (1); `--out DIR` also writes each best scheme
as text (the format `workloads.read_scheme` reads).

`--lift-333-steps N` first searches (3,3,3) over Z_T for N steps and builds
the (6,7,9) start from the best (3,3,3) scheme found (Section 3.3.2: product
with the (2,2,3:11) scheme, then extension), the way the paper lifts schemes
of small formats to larger ones.

`--explore CYCLES` runs the exploratory search of the paper's loop over a set
of formats (one population each): every cycle walks all populations, collects
each format's best scheme (population synchronisation), applies the Resize
moves to those schemes -- swap sizes with probability 1/2, then a merge with a
random best scheme, else with probability p_resize one of project (5%),
product with a random best scheme (50%), double (30%), extend (15%) -- and
re-seeds a block of walkers of any population whose best rank a result
beats.  Populations keep one format each, so the walk kernels stay
specialised; schemes move between populations between walk chunks.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import tfg
from .workloads import largest_remainder_split, naive_start

MIXED = [(2, 4, 5), (3, 3, 4), (3, 4, 5), (4, 4, 4), (4, 4, 5)]


def populations(name: str, walkers: int | None, scheme_333=None):
    """(populations, plateau length) of a named workload."""
    from . import starts
    if name == "222":
        return [((2, 2, 2), tfg.TFG_MODE_ZT, naive_start(2, 2, 2), walkers or 1024)], 10_000
    if name == "333":
        n = walkers or 65536
        return [((3, 3, 3), tfg.TFG_MODE_ZT, naive_start(3, 3, 3), n),
                ((3, 3, 3), tfg.TFG_MODE_Z2, naive_start(3, 3, 3), n)], 50_000
    if name == "333zt":
        return [((3, 3, 3), tfg.TFG_MODE_ZT, naive_start(3, 3, 3), walkers or 65536)], 50_000
    if name == "mixed":
        split = largest_remainder_split(walkers or 262144, [1, 2, 2, 4, 4])
        return [(f, tfg.TFG_MODE_ZT, naive_start(*f), n) for f, n in zip(MIXED, split)], 50_000
    if name == "large":
        return starts.large_populations(walkers or 131072, scheme_333), 50_000
    raise SystemExit(f"unknown workload {name}")


def write_scheme(path: str, fmt, scheme: np.ndarray, note: str = ""):
    m, n, p = fmt
    LU, LV = m * n, n * p
    with open(path, "w") as fh:
        if note:
            fh.write(f"# {note}\n")
        fh.write(f"format {m} {n} {p}\nrank {scheme.shape[0]}\n")
        for name, blk in (("U", scheme[:, :LU]), ("V", scheme[:, LU:LU + LV]), ("W", scheme[:, LU + LV:])):
            fh.write(name + "\n")
            for row in blk:
                fh.write(" ".join(str(int(x)) for x in row) + "\n")


def invariants(fmt, scheme, mode):
    """Type polynomial (as {"a b c": coefficient} for X^a Y^b Z^c) and rank sums
    of a scheme's factor matrices."""
    _, typ, _, sums = tfg.tfg_isotropy_invariants(fmt, scheme, mode)
    terms = tfg.polynomial_terms(typ)
    return {"type_polynomial": {f"{a} {b} {c}": v for (a, b, c), v in sorted(terms.items(), reverse=True)},
            "rank_sums": [int(x) for x in sums]}


def lift_population(W, f, max_tries: int = 256, max_nodes: int = 10**6, stop_at_first: bool = False):
    """Z_2 -> Z_T sign lifting of the best schemes of the walkers at a Z_2
    population's lowest rank (up to max_tries of them): how many lift, and the
    first ternary scheme found (stop_at_first: stop there)."""
    pop = W.pop[f]
    info, _, _ = W.read_walkers(pop["first"], pop["walkers"], slots=False, best=False)
    low = int(info["best_r"].min())
    cands = np.flatnonzero(info["best_r"] == low)[:max_tries]
    lifted, first = 0, None
    for w in cands:
        _, _, best = W.read_walkers(pop["first"] + int(w), 1, slots=False)
        s = best[0, :low]
        try:
            zt, _ = tfg.tfg_lift_signs(pop["fmt"], s, max_nodes=max_nodes)
        except tfg.TfgError:
            continue
        lifted += 1
        if first is None:
            first = zt
            if stop_at_first:
                break
    return low, len(cands), lifted, first


def run(pops, steps: int, chunk: int, seed: int, plateau: int, out_dir: str | None = None, label: str = "",
        quiet: bool = False, policy: int = 0, p_expand: float = 0.0, r_slack: int = 3):
    import torch
    params = tfg.tfg_default_params(plateau_len=plateau, walk_policy=policy,
                                    expand_thresh=min(int(p_expand * 2**32), 2**32 - 1), r_slack=r_slack)
    W = tfg.Walkers(pops, seed=seed, params=params)
    W.autotune(trial_steps=200, trial_walkers=16384)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        c = min(chunk, steps - done)
        W.walk(c)
        W.sync()
        done += c
        if not quiet:
            lows = [W.stats(f)[0]["min_best_r"] for f in range(W.n_formats)]
            print(json.dumps({"progress": done, "seconds": round(time.perf_counter() - t0, 2),
                              "lowest_ranks": lows}), flush=True)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    fails = W.verify_all()
    results = []
    for f, (fmt, mode, start, nw) in enumerate(pops):
        st, hist = W.stats(f)
        scheme, rank, walker = W.collect_best(f)
        ok = tfg.tfg_verify(fmt, scheme, mode=mode)
        res = {
            "label": label, "format": list(fmt), "mode": "Z_T" if mode == tfg.TFG_MODE_ZT else "Z_2",
            "walkers": nw, "steps_per_walker": steps, "start_rank": int(np.asarray(start).shape[0]),
            "prepared_start_rank": W.pop[f]["r0"],
            "lowest_rank": int(rank), "best_walker": int(walker),
            "walkers_at_lowest": int(hist[rank]) if rank < len(hist) else None,
            "rank_histogram": {int(k): int(v) for k, v in enumerate(hist) if v},
            "best_scheme_verified_host": bool(ok),
            "additive_complexity": int(tfg.tfg_additive_complexity(fmt, scheme)) if mode == tfg.TFG_MODE_ZT else None,
            "isotropy_invariants": invariants(fmt, scheme, mode),
            "accepted": int(st["accepted"]), "reductions": int(st["reductions"]), "plus": int(st["plus"]),
            "device_check_failures": int(fails), "seconds": round(secs, 2),
            "steps_per_s": nw * steps / secs,
        }
        if mode == tfg.TFG_MODE_Z2:
            low, tried, lifted, zt = lift_population(W, f)
            res["ternary_lifting"] = {"rank": low, "tried": tried, "lifted": lifted}
            if zt is not None:
                res["ternary_lifting"].update({"additive_complexity": int(tfg.tfg_additive_complexity(fmt, zt)),
                                               "isotropy_invariants": invariants(fmt, zt, tfg.TFG_MODE_ZT)})
                if out_dir:
                    os.makedirs(out_dir, exist_ok=True)
                    path = os.path.join(out_dir, f"lifted_{fmt[0]}x{fmt[1]}x{fmt[2]}_zt_r{low}.txt")
                    write_scheme(path, fmt, zt, f"sign lifting of a Z_2 scheme, seed {seed}, {steps} steps")
                    res["ternary_lifting"]["file"] = path
        if out_dir:
            os.makedirs(out_dir, exist_ok=True)
            tag = "zt" if mode == tfg.TFG_MODE_ZT else "z2"
            path = os.path.join(out_dir, f"best_{fmt[0]}x{fmt[1]}x{fmt[2]}_{tag}_r{rank}.txt")
            write_scheme(path, fmt, scheme, f"walker {walker}, seed {seed}, {steps} steps")
            res["file"] = path
        results.append((res, scheme))
    W.close()
    return results


EXPLORE_FORMATS = [(2, 2, 2), (2, 2, 3), (2, 2, 4), (2, 3, 3), (2, 3, 4), (3, 3, 3), (2, 4, 4), (3, 3, 4),
                   (4, 4, 4)]


def resize_move(rng, fmt, scheme, bests, p_resize=0.5):
    """One Resize move (the paper's Resize kernel) on a scheme; returns
    (format, scheme, operator) or None.  bests: {format: scheme}."""
    ops = []
    if rng.random() < 0.5:
        perm = int(rng.integers(6))
        fmt, scheme = tfg.tfg_swap_sizes(fmt, scheme, perm)
        ops.append(f"swap{perm}")
    keys = list(bests)
    other = keys[int(rng.integers(len(keys)))]
    axes = [a for a in range(3) if all(fmt[b] == other[b] for b in range(3) if b != a)]
    if axes:
        axis = axes[int(rng.integers(len(axes)))]
        try:
            f2, s2 = tfg.tfg_merge(fmt, scheme, other, bests[other], axis)
            return f2, s2, "+".join(ops + [f"merge{axis}"])
        except tfg.TfgError:
            pass
    if rng.random() >= p_resize:
        return (fmt, scheme, "+".join(ops)) if ops else None
    u = rng.random()
    try:
        if u < 0.05:
            axis = int(rng.integers(3))
            if fmt[axis] < 2:
                return None
            f2, s2 = tfg.tfg_project(fmt, scheme, axis, int(rng.integers(fmt[axis])))
            op = f"project{axis}"
        elif u < 0.55:
            other = keys[int(rng.integers(len(keys)))]
            f2, s2 = tfg.tfg_product(fmt, scheme, other, bests[other])
            op = "product"
        elif u < 0.85:
            axis = int(rng.integers(3))
            f2, s2 = tfg.tfg_double(fmt, scheme, axis)
            op = f"double{axis}"
        else:
            axis = int(rng.integers(3))
            f2, s2 = tfg.tfg_extend(fmt, scheme, axis)
            op = f"extend{axis}"
    except tfg.TfgError:
        return None
    return f2, s2, "+".join(ops + [op])


def device_resize_move(rng, W, formats, index, bests, block, next_block, p_resize=0.5):
    """One Resize move on the device (the paper's Resize kernel, applied per
    walker): a block of one population's walkers, from their best schemes,
    transformed by one operator into the next block of the population of the
    result format.  Operator choice as in resize_move: a size swap with
    probability 1/2, else a merge with another population's best when the sizes
    agree, else with probability p_resize project 5% / product 50% /
    double 30% / extend 15%.  Returns a log entry or None."""
    src = formats[int(rng.integers(len(formats)))]
    keys = list(bests)
    aux, axis, index_arg = None, 0, 0
    if rng.random() < 0.5:
        op, index_arg = tfg.TFG_RESIZE_SWAP, int(rng.integers(1, 6))
        order = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)][index_arg]
        dst = tuple(src[a] for a in order)
        name = f"swap{index_arg}"
    else:
        other = keys[int(rng.integers(len(keys)))]
        axes = [a for a in range(3) if all(src[b] == other[b] for b in range(3) if b != a)]
        if axes:
            axis = axes[int(rng.integers(len(axes)))]
            op, aux = tfg.TFG_RESIZE_MERGE, (other, bests[other])
            dst = tuple(src[b] + (other[b] if b == axis else 0) for b in range(3))
            name = f"merge{axis}"
        elif rng.random() < p_resize:
            u = rng.random()
            axis = int(rng.integers(3))
            if u < 0.05:
                if src[axis] < 2:
                    return None
                op, index_arg = tfg.TFG_RESIZE_PROJECT, int(rng.integers(src[axis]))
                dst = tuple(src[b] - (b == axis) for b in range(3))
                name = f"project{axis}"
            elif u < 0.55:
                other = keys[int(rng.integers(len(keys)))]
                op, aux = tfg.TFG_RESIZE_PRODUCT, (other, bests[other])
                dst = tuple(src[b] * other[b] for b in range(3))
                name = "product"
            elif u < 0.85:
                op = tfg.TFG_RESIZE_DOUBLE
                dst = tuple(src[b] * (2 if b == axis else 1) for b in range(3))
                name = f"double{axis}"
            else:
                op = tfg.TFG_RESIZE_EXTEND
                dst = tuple(src[b] + (b == axis) for b in range(3))
                name = f"extend{axis}"
        else:
            return None
    if dst not in index:
        return None
    ps, pd = W.pop[index[src]], W.pop[index[dst]]
    n_s, n_d = ps["walkers"], pd["walkers"]
    s_off = int(rng.integers(max(1, n_s - block + 1)))
    d_off = next_block[dst]
    if src == dst and abs(s_off - d_off) < block:
        s_off = (d_off + block) % max(1, n_s - block + 1)
        if abs(s_off - d_off) < block:
            return None
    skipped = W.resize(op, ps["first"] + s_off, pd["first"] + d_off, block, axis=axis, index=index_arg, aux=aux,
                       use_best=True)
    next_block[dst] = (d_off + block) % max(1, n_d - block + 1)
    return {"from": list(src), "to": list(dst), "op": name, "walkers": block, "skipped": skipped, "device": True}


def explore(formats, walkers: int, cycles: int, steps_per_cycle: int, seed: int, plateau: int = 50_000,
            reseed_frac: float = 0.25, p_resize: float = 0.5, moves_per_cycle: int = 8, starts: dict | None = None,
            r_slack: int = 3, quiet: bool = False, device_moves: int = 0, device_frac: float = 0.125,
            lift_z2: bool = False):
    """Exploratory search over `formats` (Z_T, one population each, naive starts
    unless `starts` gives one).  Each cycle: a walk chunk; population sync (each
    format's best collected and verified); `moves_per_cycle` Resize moves of the
    best schemes on the host, whose prepared results re-seed a block of the
    result format's walkers when they beat its best; and `device_moves` Resize
    moves on the device (device_resize_move: blocks of device_frac of a
    population, per walker).  lift_z2: a Z_2 population of every format walks
    beside the Z_T ones, and each cycle a Z_2 best below the format's Z_T best is
    lifted to Z_T signs (tfg_lift_signs) and re-seeds a block of the Z_T walkers
    (the paper's Z_2 search followed by its ternary lifting).  Returns
    (per-population results, transfer log)."""
    # one process per GPU (torch.distributed initialised): every rank runs its own
    # walkers of every format (global ids rank * len(formats) * walkers + ...), and the
    # population synchronisation takes each format's best over all ranks
    import torch.distributed as dist
    multi = dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1
    me = dist.get_rank() if multi else 0
    id_base = me * len(formats) * walkers * (2 if lift_z2 else 1)
    rng = np.random.default_rng(seed + 7919 * me)
    starts = starts or {}
    pops = [(f, tfg.TFG_MODE_ZT, starts.get(f, naive_start(*f)), walkers) for f in formats]
    if lift_z2:
        pops += [(f, tfg.TFG_MODE_Z2, np.abs(starts.get(f, naive_start(*f))).astype(np.int8), walkers)
                 for f in formats]
    W = tfg.Walkers(pops, seed=seed, params=tfg.tfg_default_params(plateau_len=plateau, r_slack=r_slack,
                                                                    walker_id_base=id_base))

    def population_sync():
        local = {}
        for f in formats:
            sch, r, w = W.collect_best(index[f])
            local[f] = (int(r), id_base + int(w), sch)
        if multi:
            from . import shard
            local = shard.sync_bests(local, {f: tfg.term_len(f) for f in formats},
                                     {f: W.pop[index[f]]["r_max"] for f in formats})
        return {f: local[f][2] for f in formats}
    index = {f: a for a, f in enumerate(formats)}             # the Z_T populations
    z2_index = {f: len(formats) + a for a, f in enumerate(formats)} if lift_z2 else {}
    block = max(1, int(walkers * reseed_frac))
    next_block = {f: 0 for f in formats}
    next_dblock = {f: 0 for f in formats}
    transfers = []
    for cycle in range(cycles):
        W.walk(steps_per_cycle)
        W.sync()
        bests = population_sync()
        for _ in range(moves_per_cycle):
            src = formats[int(rng.integers(len(formats)))]
            out = resize_move(rng, src, bests[src], bests, p_resize)
            if out is None:
                continue
            f2, s2, op = out
            f2 = tuple(f2)
            if f2 not in index:
                continue
            prepared = tfg.tfg_prepare(f2, s2)
            if prepared.shape[0] >= bests[f2].shape[0] or prepared.shape[0] > W.pop[index[f2]]["r_max"]:
                continue
            first = W.pop[index[f2]]["first"] + next_block[f2]
            W.reseed(first, block, prepared)
            next_block[f2] = (next_block[f2] + block) % max(1, walkers - block + 1)
            bests[f2] = prepared
            transfers.append({"cycle": cycle, "from": list(src), "to": list(f2), "op": op,
                              "rank": int(prepared.shape[0])})
            if not quiet:
                print(json.dumps({"transfer": transfers[-1]}), flush=True)
        for f, zf in z2_index.items():
            low = W.stats(zf)[0]["min_best_r"]
            if low >= bests[f].shape[0]:
                continue
            _, _, _, zt = lift_population(W, zf, max_tries=32, stop_at_first=True)
            if zt is None:
                continue
            prepared = tfg.tfg_prepare(f, zt)
            if prepared.shape[0] >= bests[f].shape[0] or prepared.shape[0] > W.pop[index[f]]["r_max"]:
                continue
            first = W.pop[index[f]]["first"] + next_block[f]
            W.reseed(first, block, prepared)
            next_block[f] = (next_block[f] + block) % max(1, walkers - block + 1)
            bests[f] = prepared
            transfers.append({"cycle": cycle, "from": list(f), "to": list(f), "op": "lift",
                              "rank": int(prepared.shape[0])})
            if not quiet:
                print(json.dumps({"transfer": transfers[-1]}), flush=True)
        dblock = max(1, int(walkers * device_frac))
        for _ in range(device_moves):
            t = device_resize_move(rng, W, formats, index, bests, dblock, next_dblock, p_resize)
            if t is not None:
                t["cycle"] = cycle
                transfers.append(t)
                if not quiet:
                    print(json.dumps({"transfer": t}), flush=True)
        if not quiet and me == 0:
            print(json.dumps({"cycle": cycle, "best_ranks": {"x".join(map(str, f)): int(bests[f].shape[0])
                                                              for f in formats}}), flush=True)
    fails = W.verify_all()
    results = []
    for f in formats:
        sch, r, w = W.collect_best(index[f])
        results.append({"format": list(f), "mode": "Z_T", "lowest_rank": int(r), "best_walker": int(w),
                        "best_scheme_verified_host": bool(tfg.tfg_verify(f, sch)),
                        "additive_complexity": int(tfg.tfg_additive_complexity(f, sch)),
                        "isotropy_invariants": invariants(f, sch, tfg.TFG_MODE_ZT),
                        "device_check_failures": int(fails)})
    for f, zf in z2_index.items():
        # the Z_2 populations: their own lowest rank and how many of the walkers at
        # that rank lift to Z_T signs
        sch, r, w = W.collect_best(zf)
        low, tried, lifted, _ = lift_population(W, zf, max_tries=32)
        results.append({"format": list(f), "mode": "Z_2", "lowest_rank": int(r), "best_walker": int(w),
                        "best_scheme_verified_host": bool(tfg.tfg_verify(f, sch, tfg.TFG_MODE_Z2)),
                        "lift": {"rank": int(low), "tried": int(tried), "lifted": int(lifted)},
                        "device_check_failures": int(fails)})
    W.close()
    return results, transfers


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="333")
    ap.add_argument("--walkers", type=int, default=None)
    ap.add_argument("--steps", type=float, default=1e6)
    ap.add_argument("--chunk", type=int, default=100_000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--plateau", type=int, default=None)
    ap.add_argument("--lift-333-steps", type=float, default=0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--walk-policy", type=int, default=0,
                    help="0: plus transitions on plateaus; 1: Algorithm 1 expansions (plus or split)")
    ap.add_argument("--p-expand", type=float, default=0.0, help="walk policy 1: expansion probability after a flip")
    ap.add_argument("--r-slack", type=int, default=3, help="slots per walker beyond the start rank")
    ap.add_argument("--explore", type=int, default=0, help="exploratory search: number of walk + resize cycles")
    ap.add_argument("--formats", default=None,
                    help="exploratory search: formats as m x n x p list, e.g. 2x2x2,3x3x3 (default: nine up to 4x4x4)")
    ap.add_argument("--lift-z2", action="store_true",
                    help="exploratory search: Z_2 populations beside the Z_T ones, lifted to Z_T each cycle")
    ap.add_argument("--device-moves", type=int, default=0,
                    help="exploratory search: Resize moves per cycle on the device (blocks of walkers)")
    ap.add_argument("--quiet", action="store_true")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    if args.explore > 0:
        fmts = EXPLORE_FORMATS if not args.formats else \
            [tuple(int(x) for x in f.split("x")) for f in args.formats.split(",")]
        res, transfers = explore(fmts, args.walkers or 16384, args.explore, int(args.steps), args.seed,
                                 plateau=args.plateau or 50_000, r_slack=args.r_slack, quiet=args.quiet,
                                 device_moves=args.device_moves, lift_z2=args.lift_z2)
        for r in res:
            print(json.dumps(r), flush=True)
        print(json.dumps({"transfers": len(transfers)}), flush=True)
        return
    scheme_333 = None
    if args.workload == "large" and args.lift_333_steps > 0:
        pops, plateau = populations("333zt", None)
        (res, scheme_333), = run(pops, int(args.lift_333_steps), args.chunk, args.seed, plateau, args.out,
                                 "lift (3,3,3)", args.quiet, args.walk_policy, args.p_expand, args.r_slack)
        print(json.dumps(res), flush=True)
    pops, plateau = populations(args.workload, args.walkers, scheme_333)
    for res, _ in run(pops, int(args.steps), args.chunk, args.seed, args.plateau or plateau, args.out,
                      args.workload, args.quiet, args.walk_policy, args.p_expand, args.r_slack):
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
