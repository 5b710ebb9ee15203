"""Window-mode walks (the learned proposal's step) against the oracle: uniform
policy bit-exact; learned policy replayed from the logged choices bit-exact;
window features bit-exact; network scores and greedy choices within the
tensor-core tolerance."""
import os

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2511_20317_gb300 import tfg
from paper_2511_20317_gb300.workloads import naive_start

pytestmark = pytest.mark.gpu
THREADS = len(os.sched_getaffinity(0))
FIELDS = ["r", "best_r", "t", "plateau", "best_t", "digest", "accepted", "rejected", "nocand", "drops",
          "merges", "plus", "reductions"]


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_2511_20317_gb300 import _build
    _build.build()
    tfg.lib()


def device_params(p):
    import torch
    return torch.from_numpy(np.frombuffer(p.blob(), dtype=np.uint8).copy()).cuda()


def assert_parity(W, ref, n, label):
    info, slots, best = W.read_walkers(0, n)
    assert (ref.info["debug_failures"] == 0).all(), label
    for w in range(n):
        for f in FIELDS:
            assert info[f][w] == ref.info[f][w], f"{label} walker {w}: {f} gpu={info[f][w]} oracle={ref.info[f][w]}"
        r, br = ref.info["r"][w], ref.info["best_r"][w]
        assert np.array_equal(slots[w, :r], ref.slots[w, :r]), f"{label} walker {w} slots"
        assert np.array_equal(best[w, :br], ref.best[w, :br]), f"{label} walker {w} best"


# window capacities of the apply kernel: 12 (32-bit words), 32, 64, 72 and 88 (64-bit words)
CASES = [((2, 2, 2), 300, 3000, 200), ((3, 3, 3), 160, 1500, 300), ((3, 4, 5), 70, 400, 100),
         ((4, 4, 4), 70, 400, 100), ((4, 4, 5), 40, 300, 100)]


@pytest.mark.parametrize("fmt,nw,steps,L", CASES)
def test_window_uniform_parity(fmt, nw, steps, L):
    start = naive_start(*fmt)
    W = tfg.Walkers([(fmt, 0, start, nw)], seed=5, params=tfg.tfg_default_params(plateau_len=L))
    W.walk_window(steps, policy=0)
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=5, plateau_len=L).walk_window(steps, threads=THREADS)
    assert_parity(W, ref, nw, f"window-uniform {fmt}")
    assert W.verify_all() == 0


@pytest.mark.parametrize("fmt,nw,steps,L", CASES[1:])
def test_window_learned_replay(fmt, nw, steps, L):
    """The learned policy's decisions are replayed by the oracle from the
    logged window indices: every trajectory matches bit for bit."""
    start = naive_start(*fmt)
    p = mlp.Params.random(np.random.default_rng(11))
    W = tfg.Walkers([(fmt, 0, start, nw)], seed=6, params=tfg.tfg_default_params(plateau_len=L))
    ch = W.walk_window(steps, policy=1, mlp_params=device_params(p), eps_thresh=int(0.2 * 2**32),
                       record_choices=True).cpu().numpy()
    assert (ch >= -1).all()
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=6, plateau_len=L).walk_window(
        steps, policy=1, choices=ch.T, threads=THREADS)
    assert_parity(W, ref, nw, f"window-learned {fmt}")


@pytest.mark.parametrize("policy", [0, 1])
def test_window_full_size_sampled(policy):
    """The learned-proposal workload at its full size: (4,4,4) naive, 262144 walkers,
    window steps with the uniform (0) or the learned (1, eps 0.05, a random network)
    choice; 16 walkers spread over the population replayed by the oracle (the
    learned ones from their logged window indices)."""
    fmt, nw, steps, L = (4, 4, 4), 262144, 60, 50_000
    start = naive_start(*fmt)
    W = tfg.Walkers([(fmt, 0, start, nw)], seed=8, params=tfg.tfg_default_params(plateau_len=L))
    if policy == 1:
        p = mlp.Params.random(np.random.default_rng(5))
        ch = W.walk_window(steps, policy=1, mlp_params=device_params(p), eps_thresh=int(0.05 * 2**32),
                           record_choices=True).cpu().numpy()
    else:
        W.walk_window(steps, policy=0)
    W.sync()
    ids = np.linspace(0, nw - 1, 16).astype(int)
    rows = [W.read_walkers(int(w), 1) for w in ids]
    info = np.concatenate([x[0] for x in rows])
    slots = np.concatenate([x[1] for x in rows])
    best = np.concatenate([x[2] for x in rows])
    ref = oracle.Walkers(fmt, start, ids, seed=8, plateau_len=L)
    if policy == 1:
        ref.walk_window(steps, policy=1, choices=np.ascontiguousarray(ch[:, ids].T), threads=THREADS)
    else:
        ref.walk_window(steps, threads=THREADS)
    assert (ref.info["accepted"] > 0).any()
    for a in range(ids.size):
        for f in FIELDS:
            assert info[f][a] == ref.info[f][a], f"walker {ids[a]}: {f} gpu={info[f][a]} oracle={ref.info[f][a]}"
        r, br = ref.info["r"][a], ref.info["best_r"][a]
        assert np.array_equal(slots[a, :r], ref.slots[a, :r]) and np.array_equal(best[a, :br], ref.best[a, :br])
    W.close()


@pytest.mark.parametrize("fmt", [(3, 3, 3), (4, 4, 4)])
def test_window_features_scores_and_choice(fmt):
    """One learned step from a walked state: the window (candidate rows, their
    info words and the features tfg_window_dump writes) equals the oracle's;
    the scores the fused tensor-core kernel computes from the candidate rows
    match the float64 network on the oracle's features within the bf16 bound;
    exploit steps pick a candidate whose reference score is the maximum up to
    that bound; explore steps (x3 < eps) pick mulhi(x1, K)."""
    nw, eps = 96, int(0.25 * 2**32)
    start = naive_start(*fmt)
    W = tfg.Walkers([(fmt, 0, start, nw)], seed=9, params=tfg.tfg_default_params(plateau_len=150))
    W.walk_window(300, policy=0)
    info0, slots0, _ = W.read_walkers(0, nw)
    feat, rows, kwin = (b.cpu() for b in W.window_dump())
    feat, rows, kwin = feat.float().numpy(), rows.numpy().view(np.uint32), kwin.numpy()
    p = mlp.Params.random(np.random.default_rng(4))
    ch = W.walk_window(1, policy=1, mlp_params=device_params(p), eps_thresh=eps, record_choices=True)
    ch = ch.cpu().numpy()[0]
    rows2, score, kwin2 = (b.cpu().numpy() for b in W.window_buffers())
    assert np.array_equal(kwin2, kwin)
    for w in range(nw):
        r, br, t, wid = int(info0["r"][w]), int(info0["best_r"][w]), int(info0["t"][w]), int(info0["walker_id"][w])
        x = oracle.philox4x32_10([t & 0xFFFFFFFF, t >> 32, wid, 0], [9, 0])
        i0 = (int(x[0]) * r) >> 32
        f_ref, c_ref = oracle.window_features(fmt, slots0[w, :r], br, i0)
        K = f_ref.shape[0]
        assert kwin[w] == K
        assert np.array_equal(feat[w, :K], f_ref) and not feat[w, K:].any()
        d, info = rows[w, :K, 0], rows[w, :K, 1]
        assert np.array_equal(rows2[w, :K].view(np.uint32), rows[w, :K])
        got = np.stack([d & 1023, (d >> 10) & 3, (d >> 12) & 1023, np.where((d >> 22) & 1, -1, 1), (d >> 23) & 1], 1)
        assert np.array_equal(got, c_ref)
        assert np.array_equal(info & 255, f_ref[:, 18]) and np.array_equal(info >> 8, f_ref[:, 24])
        y, cache = mlp.forward(p, f_ref)
        path = np.abs(p.W2) @ np.abs(p.w3)
        bound = 2 * ((np.abs(cache[2]) * 2.0 ** -8) * path).max(axis=1) + 1e-5 * (1 + np.abs(y))
        assert (np.abs(score[w, :K] - y) <= bound).all()
        if K == 0:
            assert ch[w] == -1
        elif int(x[3]) < eps:
            assert ch[w] == (int(x[1]) * K) >> 32
        else:
            assert y[ch[w]] >= y.max() - 2 * bound.max()


def test_transition_log_equals_the_oracle_log():
    """The device's training log, entry by entry, against the log the oracle's
    window walk writes for the same walkers: every rank-lowering step with label
    1 and the label-0 steps sampled by Philox sub-stream 256, each with the chosen
    candidate's features, walker id and step (entries sorted by walker and step;
    the device appends them in arrival order)."""
    fmt, nw, steps, L = (3, 3, 3), 256, 700, 200
    neg = int(0.02 * 2**32)
    start = naive_start(*fmt)
    W = tfg.Walkers([(fmt, 0, start, nw)], seed=3, params=tfg.tfg_default_params(plateau_len=L))
    log = tfg.TransitionLog(nw * steps, neg_thresh=neg)
    W.walk_window(steps, policy=0, log=log)
    W.sync()
    st, _ = W.stats()
    assert int(log.count.item()) <= log.capacity
    e = log.read()
    e = e[np.lexsort((e["step"], e["walker_id"]))]
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=3, plateau_len=L).walk_window(
        steps, threads=THREADS, log_neg_thresh=neg)
    w_idx, t_idx = np.nonzero(ref.log_label >= 0)          # row-major: sorted by walker, then step
    assert e.size == w_idx.size, (e.size, w_idx.size)
    assert np.array_equal(e["walker_id"], w_idx.astype(np.uint32))
    assert np.array_equal(e["step"], t_idx.astype(np.uint32))
    assert np.array_equal(e["label"], ref.log_label[w_idx, t_idx].astype(np.float32))
    want_feat = mlp.bf16_bits(ref.log_feat[w_idx, t_idx].astype(np.float32))
    assert np.array_equal(e["feat"], want_feat)
    assert int((e["label"] == 1).sum()) == st["reductions"]
    assert (e["label"] == 0).sum() > 0


@pytest.mark.parametrize("H", [2, 8])
def test_transition_log_with_horizon_equals_the_oracle_log(H):
    """H-step horizon: every rank-lowering step logs the chosen candidates of
    its last H steps (since the previous rank-lowering step) with label 1.  The
    device walks in two calls, so the per-walker rings carry over between them;
    the oracle's log comes from one walk of all the steps."""
    fmt, nw, steps, L = (3, 3, 3), 256, 700, 200
    neg = int(0.02 * 2**32)
    start = naive_start(*fmt)
    W = tfg.Walkers([(fmt, 0, start, nw)], seed=3, params=tfg.tfg_default_params(plateau_len=L))
    log = tfg.TransitionLog(nw * steps, neg_thresh=neg, horizon=H)
    W.walk_window(300, policy=0, log=log)
    W.walk_window(steps - 300, policy=0, log=log)
    W.sync()
    st, _ = W.stats()
    assert int(log.count.item()) <= log.capacity
    e = log.read()
    e = e[np.lexsort((e["label"], e["step"], e["walker_id"]))]
    ref = oracle.Walkers(fmt, start, np.arange(nw), seed=3, plateau_len=L).walk_window(
        steps, threads=THREADS, log_neg_thresh=neg)
    wid, stp, lab, feat = oracle.horizon_log(ref.log_label, ref.log_feat, ref.log_chosen, np.arange(nw), H)
    assert e.size == wid.size, (e.size, wid.size)
    assert np.array_equal(e["walker_id"], wid.astype(np.uint32))
    assert np.array_equal(e["step"], stp.astype(np.uint32))
    assert np.array_equal(e["label"], lab)
    assert np.array_equal(e["feat"], mlp.bf16_bits(feat.astype(np.float32)))
    assert (e["label"] == 1).sum() > st["reductions"]       # the horizon adds the steps before each reduction


def test_transition_log_horizon_out_of_range_is_rejected():
    fmt = (2, 2, 2)
    W = tfg.Walkers([(fmt, 0, naive_start(*fmt), 8)], seed=1)
    with pytest.raises(tfg.TfgError):
        W.walk_window(1, policy=0, log=tfg.TransitionLog(64, horizon=65))
    W.walk_window(1, policy=0, log=tfg.TransitionLog(64, horizon=64))
    W.sync()
