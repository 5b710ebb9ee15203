"""Learned flip proposal: data collection, device training and the A/B test
against the uniform proposal over the same candidate windows.

Every step of the walk and of the network runs in libtfg's kernels; this module
only sequences them.  Usage:

    python -m paper_2511_20317_gb300.learned --ab      # collect, train, compare
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import tfg
from .workloads import MIXED_FORMATS, naive_start

TRAIN_FORMATS = [(2, 2, 2), (3, 3, 3)] + MIXED_FORMATS   # the formats of the uniform workloads
EVAL_FORMATS = [(4, 4, 4), (3, 4, 5)]


def init_params(seed: int = 0):
    """He-style random parameter blob (device uint8 tensor)."""
    import torch
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / 32), (32, 128)).astype(np.float32)
    W2 = rng.normal(0, np.sqrt(2.0 / 128), (128, 128)).astype(np.float32)
    b1 = np.zeros(128, np.float32)
    b2 = np.zeros(128, np.float32)
    w3 = rng.normal(0, np.sqrt(1.0 / 128), 128).astype(np.float32)
    parts = [_bf16_bits(W1), _bf16_bits(W2), b1.tobytes(), b2.tobytes(), w3.tobytes(),
             np.zeros(4, np.float32).tobytes()]
    blob = np.frombuffer(b"".join(parts), dtype=np.uint8).copy()
    assert blob.size == tfg.tfg_mlp_param_bytes()
    return torch.from_numpy(blob).cuda()


def _bf16_bits(a: np.ndarray) -> bytes:
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r.tobytes()


def collect(formats=TRAIN_FORMATS, walkers=4096, steps=4000, seed=100, neg_rate=0.01, plateau=None, horizon=1):
    """Window-uniform walks with transition logging: the chosen candidates of
    the last `horizon` steps before every rank-lowering step (label 1; horizon
    1: that step's alone) and a neg_rate sample of the others (label 0).
    plateau None: the configurations' plateau lengths (1e4 for (2,2,2), 5e4
    for the others)."""
    entries = []
    for k, fmt in enumerate(formats):
        L = plateau if plateau is not None else (10_000 if tuple(fmt) == (2, 2, 2) else 50_000)
        W = tfg.Walkers([(fmt, 0, naive_start(*fmt), walkers)], seed=seed + k,
                        params=tfg.tfg_default_params(plateau_len=L))
        log = tfg.TransitionLog(walkers * steps // 20 + 100000, neg_thresh=int(neg_rate * 2**32), horizon=horizon)
        W.walk_window(steps, policy=0, log=log)
        entries.append(canonical_order(log.read()))
        W.close()
    return np.concatenate(entries)


def canonical_order(entries):
    """Log entries sorted by walker, step and label: the device appends them in
    arrival order, which differs from run to run, and the training batches are
    drawn from positions in this array."""
    return entries[np.lexsort((entries["label"], entries["step"], entries["walker_id"]))]


def train(entries, params=None, epochs=30, batch=8192, lr=2e-3, seed=0):
    """Adam on the device, class-balanced weighted logistic loss."""
    import torch
    if params is None:
        params = init_params(seed)
    rng = np.random.default_rng(seed)
    feats = torch.from_numpy(entries["feat"].view(np.int16).copy()).cuda().view(torch.bfloat16)
    labels = torch.from_numpy(entries["label"].astype(np.float32)).cuda()
    n = labels.numel()
    pos = float(labels.sum().item())
    neg = n - pos
    tr = tfg.MlpTrainer(params)
    history = []
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        for b0 in range(0, n - batch + 1 if n >= batch else 1, batch):
            idx = perm[b0:b0 + batch]
            x = feats[idx].contiguous()
            y = labels[idx].contiguous()
            p_b = float(y.sum().item())
            n_b = y.numel() - p_b
            w = torch.where(y > 0, 0.5 / max(p_b, 1.0), 0.5 / max(n_b, 1.0)).float().contiguous()
            tr.step(x, y, w, lr)
        history.append(tr.loss())
    return params, {"samples": n, "positives": pos, "negatives": neg, "loss": history}


def evaluate(fmt, policy, params=None, walkers=262144, steps=1500, seed=0, eps=0.05, plateau=50_000,
             seconds=None, chunk=100):
    """One arm of the A/B: window-mode walks from the naive scheme for `steps`
    steps per walker, or (seconds given) for as many whole chunks of steps as
    fit in that wall time.  Returns the lowest rank, the final best-rank
    histogram, the net rank descent (start rank - mean best rank), reductions
    per 1e9 applied flips, steps/s; every walker's best scheme is verified."""
    import torch
    start = naive_start(*fmt)
    W = tfg.Walkers([(fmt, 0, start, walkers)], seed=seed, params=tfg.tfg_default_params(plateau_len=plateau))
    r0 = W.pop[0]["r0"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    if seconds is None:
        W.walk_window(steps, policy=policy, mlp_params=params, eps_thresh=int(eps * 2**32))
        W.sync()
        done = steps
    else:
        while time.perf_counter() - t0 < seconds:
            W.walk_window(chunk, policy=policy, mlp_params=params, eps_thresh=int(eps * 2**32))
            W.sync()
            done += chunk
    dt = time.perf_counter() - t0
    st, hist = W.stats()
    fails = W.verify_all()
    scheme, rank, _ = W.collect_best(0)
    W.close()
    ranks = np.arange(hist.size)
    mean_best = float((hist * ranks).sum() / max(hist.sum(), 1))
    return {"steps_per_walker": done, "seconds": dt, "lowest_rank": st["min_best_r"],
            "mean_best_rank": mean_best, "net_descent": r0 - mean_best,
            "reductions_per_1e9_applied": st["reductions"] / max(st["accepted"], 1) * 1e9,
            "applied_frac": st["accepted"] / max(st["steps"], 1), "steps_per_s": st["steps"] / dt,
            "verify_failures": fails, "collected_verified": bool(tfg.tfg_verify(fmt, scheme)),
            "rank_hist": {int(k): int(v) for k, v in enumerate(hist) if v}}


def _summary(runs, keys=("net_descent", "mean_best_rank", "lowest_rank", "reductions_per_1e9_applied",
                          "steps_per_s", "steps_per_walker")):
    out = {}
    for k in keys:
        v = np.array([r[k] for r in runs], dtype=np.float64)
        ci = float(1.96 * v.std(ddof=1) / np.sqrt(v.size)) if v.size > 1 else None
        out[k] = {"mean": float(v.mean()), "ci95": ci}
    hist = {}
    for r in runs:
        for k, v in r["rank_hist"].items():
            hist[k] = hist.get(k, 0) + v
    out["rank_hist_all_seeds"] = {int(k): int(v) for k, v in sorted(hist.items())}
    out["lowest_rank_any_seed"] = int(min(r["lowest_rank"] for r in runs))
    out["verify_failures"] = int(sum(r["verify_failures"] for r in runs))
    out["collected_verified"] = all(r["collected_verified"] for r in runs)
    return out


def _beats(a, b, key, higher_better=True):
    """a beats b on key when their 95% intervals do not overlap in a's favour."""
    ma, ca = a[key]["mean"], a[key]["ci95"] or 0.0
    mb, cb = b[key]["mean"], b[key]["ci95"] or 0.0
    return (ma - ca > mb + cb) if higher_better else (ma + ca < mb - cb)


def ab_test(params, formats=EVAL_FORMATS, seeds=(0, 1, 2, 3, 4), walkers=262144, steps=1500, eps=0.05,
            plateau=50_000, seed_base=1000):
    """Learned against uniform over the same candidate windows: per format and
    evaluation seed (disjoint from the training seeds), the learned arm for
    `steps` steps per walker, the uniform arm for the same steps (equal step
    budget) and for the learned arm's wall time (equal time).  Net measures:
    rank descent and lowest rank with 95% intervals over the seeds.  The
    evaluation walks use seeds seed_base + s."""
    out = {}
    for fmt in formats:
        learned, uniform, uniform_t = [], [], []
        for s in seeds:
            sd = seed_base + s
            l = evaluate(fmt, 1, params, walkers=walkers, steps=steps, seed=sd, eps=eps, plateau=plateau)
            learned.append(l)
            uniform.append(evaluate(fmt, 0, None, walkers=walkers, steps=steps, seed=sd, plateau=plateau))
            uniform_t.append(evaluate(fmt, 0, None, walkers=walkers, seed=sd, plateau=plateau, seconds=l["seconds"]))
        res = {"equal_steps": {"learned": _summary(learned), "uniform": _summary(uniform)},
               "equal_time": {"learned": _summary(learned), "uniform": _summary(uniform_t)}}
        eq, et = res["equal_steps"], res["equal_time"]
        res["learned_beats_uniform"] = {
            "net_descent_equal_steps": _beats(eq["learned"], eq["uniform"], "net_descent"),
            "net_descent_equal_time": _beats(et["learned"], et["uniform"], "net_descent"),
            "reductions_per_1e9_applied_equal_steps": _beats(eq["learned"], eq["uniform"],
                                                             "reductions_per_1e9_applied")}
        out["x".join(map(str, fmt))] = res
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ab", action="store_true")
    ap.add_argument("--walkers", type=int, default=262144)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--collect-walkers", type=int, default=4096)
    ap.add_argument("--collect-steps", type=int, default=4000)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--seeds", type=int, default=5)
    ap.add_argument("--horizon", type=int, default=1, help="label-1 horizon of the training log (steps)")
    ap.add_argument("--eval-seed-base", type=int, default=1000)
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    e = collect(walkers=args.collect_walkers, steps=args.collect_steps, horizon=args.horizon)
    t1 = time.perf_counter()
    params, info = train(e, epochs=args.epochs)
    t2 = time.perf_counter()
    res = ab_test(params, seeds=tuple(range(args.seeds)), walkers=args.walkers, steps=args.steps,
                  seed_base=args.eval_seed_base)
    t3 = time.perf_counter()
    print(json.dumps({"train": {k: v for k, v in info.items() if k != "loss"}, "loss_first_last":
                      [info["loss"][0], info["loss"][-1]], "ab": res,
                      "seconds": {"collect": t1 - t0, "train": t2 - t1, "ab": t3 - t2}}))


if __name__ == "__main__":
    main()
