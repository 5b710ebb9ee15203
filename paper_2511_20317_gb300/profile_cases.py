"""Single-launch cases of the hot kernels, sized for profiler captures.

    python -m paper_2511_20317_gb300.profile_cases --case walk_zt333
    python -m paper_2511_20317_gb300.profile_cases --case all

Each case builds its inputs, runs one warm-up launch of a different size, then
the profiled launch, and prints its CUDA-event time.
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import tfg
from .workloads import naive_start


def _timed(fn):
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e)


def walk(fmt, mode, walkers=65536, steps=2000, start=None, mapping=0):
    start = naive_start(*fmt) if start is None else start
    params = tfg.tfg_default_params(plateau_len=50_000, use_graph=0)
    params.mapping = mapping
    W = tfg.Walkers([(fmt, mode, start, walkers)], seed=0, params=params)
    W.walk(16).sync()
    ms = _timed(lambda: W.walk(steps))
    return {"walkers": walkers, "steps": steps, "ms": ms, "steps_per_s": walkers * steps / ms * 1e3,
            "mapping": (W.pop[0]["lanes"], W.pop[0]["slots_per_lane"])}


def walk_large(which, walkers=16384, steps=300):
    from . import starts
    fmt, start = {"4512": starts.start_4_5_12, "5610": starts.start_5_6_10, "679": starts.start_6_7_9}[which]()
    return walk(fmt, 0, walkers=walkers, steps=steps, start=start)


def resize(op_name="extend", walkers=65536):
    """Device resize of a whole (3,3,3) population (walked 2000 steps) into a
    (3,3,4) population (extend along p) or a (3,3,3) population (size swap)."""
    src = (3, 3, 3)
    op, dst, kw = {"extend": (tfg.TFG_RESIZE_EXTEND, (3, 3, 4), {"axis": 2}),
                   "swap": (tfg.TFG_RESIZE_SWAP, (3, 3, 3), {"index": 3})}[op_name]
    pops = [(src, 0, naive_start(*src), walkers), (dst, 0, naive_start(*dst), walkers)]
    W = tfg.Walkers(pops, seed=0, params=tfg.tfg_default_params(plateau_len=50_000, r_slack=8, use_graph=0))
    W.walk(2000).sync()
    first = W.pop[1]["first"]
    W.resize(op, 0, first, walkers, **kw)
    t0 = time.perf_counter()   # the call is synchronous: host plan, staging, kernel
    W.resize(op, 0, first, walkers, **kw)
    ms = (time.perf_counter() - t0) * 1e3
    return {"walkers": walkers, "ms": ms, "walkers_per_s": walkers / ms * 1e3}


def mlp_score(rows=1 << 20):
    import torch
    rng = np.random.default_rng(0)
    from .learned import init_params
    params = init_params(0)
    x = torch.from_numpy(rng.integers(0, 9, size=(rows, 32)).astype(np.float32)).cuda().bfloat16()
    tfg.tfg_mlp_score(params, x[:1024])
    ms = _timed(lambda: tfg.tfg_mlp_score(params, x))
    flops = rows * 2 * (32 * 128 + 128 * 128 + 128)
    return {"rows": rows, "ms": ms, "tflops": flops / ms / 1e9}


def mlp_grad(rows=1 << 18):
    import torch
    rng = np.random.default_rng(1)
    from .learned import init_params
    params = init_params(1)
    x = torch.from_numpy(rng.integers(0, 9, size=(rows, 32)).astype(np.float32)).cuda().bfloat16()
    lab = torch.from_numpy((rng.random(rows) < 0.1).astype(np.float32)).cuda()
    wt = torch.full((rows,), 1.0 / rows, device="cuda")
    tfg.tfg_mlp_grad(params, x[:1024], lab[:1024], wt[:1024])
    ms = _timed(lambda: tfg.tfg_mlp_grad(params, x, lab, wt))
    # forward 2 products, backward 3 (dH1, dW2, dW1)
    flops = rows * 2 * (32 * 128 + 128 * 128) + rows * 2 * (128 * 128 + 128 * 128 + 128 * 32)
    return {"rows": rows, "ms": ms, "tflops": flops / ms / 1e9}


def window(fmt=(4, 4, 4), walkers=16384, policy=0, steps=1):
    """Window-mode steps: uniform (policy 0) or learned (1, a random network; its
    scoring is the fused feature + MLP kernel over 2 x 128-row tiles per walker)."""
    from .learned import init_params
    params = init_params(0) if policy == 1 else None
    W = tfg.Walkers([(fmt, 0, naive_start(*fmt), walkers)], seed=0, params=tfg.tfg_default_params(plateau_len=50_000))
    W.walk_window(2, policy=policy, mlp_params=params)
    W.sync()
    ms = _timed(lambda: W.walk_window(steps, policy=policy, mlp_params=params))
    out = {"walkers": walkers, "policy": policy, "ms_per_window_step": ms / steps,
           "steps_per_s": walkers * steps / ms * 1e3}
    if policy == 1:
        _, _, kwin = W.window_buffers()
        rows = int(kwin.sum().item())          # scored rows of the last step (tiles of 128 rows: more)
        out["scored_rows_per_step"] = rows
        out["score_tflops_per_step_upper"] = rows * 2 * (32 * 128 + 128 * 128 + 128) / (ms / steps) / 1e9
    return out


CASES = {
    "walk_zt333": lambda: walk((3, 3, 3), 0),
    "walk_z2333": lambda: walk((3, 3, 3), 1),
    "walk_zt222": lambda: walk((2, 2, 2), 0),
    "walk_zt445": lambda: walk((4, 4, 5), 0, walkers=80660, steps=500),
    "walk_zt245": lambda: walk((2, 4, 5), 0, walkers=20165, steps=1000),
    "walk_zt334": lambda: walk((3, 3, 4), 0, walkers=40330, steps=1000),
    "walk_zt345": lambda: walk((3, 4, 5), 0, walkers=40330, steps=1000),
    "walk_zt444": lambda: walk((4, 4, 4), 0, walkers=80660, steps=500),
    "walk_zt4512": lambda: walk_large("4512"),
    "walk_zt5610": lambda: walk_large("5610"),
    "walk_zt679": lambda: walk_large("679"),
    "walk_zt982": lambda: walk((9, 8, 2), 0, walkers=16384, steps=300),
    "walk_zt1111": lambda: walk((11, 11, 1), 0, walkers=16384, steps=300),
    "walk_z2982": lambda: walk((9, 8, 2), 1, walkers=16384, steps=300),
    "resize_extend_333": lambda: resize("extend"),
    "resize_swap_333": lambda: resize("swap"),
    "mlp_score": mlp_score,
    "mlp_score_33m": lambda: mlp_score(rows=1 << 25),
    "mlp_grad": mlp_grad,
    "window_444": window,
    "window_444_262k": lambda: window(walkers=262144, steps=20),
    "window_444_learned": lambda: window(policy=1),
    "window_444_learned_262k": lambda: window(walkers=262144, policy=1, steps=20),
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="all")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    names = list(CASES) if args.case == "all" else args.case.split(",")
    for n in names:
        t0 = time.perf_counter()
        res = CASES[n]()
        print(n, res, f"wall {time.perf_counter() - t0:.2f}s", flush=True)


if __name__ == "__main__":
    main()
