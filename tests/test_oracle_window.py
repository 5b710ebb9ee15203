"""Pins of the oracle's window mode (the step the learned proposal acts on),
its training log and its Adam step, against things other than the oracle's
own window code:

* the window is the concatenation, over terms i0, i0+1, ... (mod r), of the
  try_flip candidate lists (which test_oracle_walk pins by brute force),
  truncated at the window capacity, also in the middle of a term;
* every one of the 32 features equals a direct numpy restatement of its
  definition, and on hand-built states equals values counted by hand;
* the training log holds exactly the rank-lowering steps (label 1) and the
  other steps whose Philox sub-stream 256 draw (Philox pinned by its
  known-answer vectors) is below the threshold (label 0), each with the
  features of the chosen candidate on the state before the step;
* Adam (Kingma & Ba) against its closed forms and torch.optim.Adam.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2511_20317_gb300.workloads import naive_start

FORMATS = [(2, 2, 2), (3, 3, 3), (2, 3, 4), (4, 4, 4)]


def walked_states(fmt, n=6, steps=400, seed=7):
    """States reached by oracle walks (various ranks; some after plus transitions)."""
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(n), seed=seed, plateau_len=60).walk(steps, threads=2)
    return [(W.scheme(w), int(W.info["best_r"][w])) for w in range(n)]


def candidate_rows(fmt, scheme, i):
    return [(i, int(X), int(j), int(s), int(rho)) for X, j, s, rho in oracle.enumerate_candidates(fmt, scheme, i)]


@pytest.mark.parametrize("fmt", FORMATS)
def test_window_is_the_concatenation_of_term_candidate_lists(fmt):
    for scheme, best_r in walked_states(fmt):
        r = scheme.shape[0]
        for i0 in sorted({0, r // 2, r - 1}):
            full = []
            for q in range(r):
                full += candidate_rows(fmt, scheme, (i0 + q) % r)
            for W in (oracle.WINDOW, 7, 5, 1):   # odd capacities cut a term's candidate pairs in the middle
                _, cand = oracle.window_features(fmt, scheme, best_r, i0, W=W)
                want = full[:W]
                assert [tuple(int(v) for v in c) for c in cand] == want, (fmt, i0, W)


def features_by_definition(fmt, scheme, r, best_r, i, X, j, s, rho, k_i, q):
    """The 32 features of candidate (X, j, s, rho) of term i, restated from their
    definition with plain integer arrays."""
    m, n, p = fmt
    L = [m * n, n * p, p * m]
    off = [0, L[0], L[0] + L[1]]
    fac = lambda t, f: scheme[t, off[f]:off[f] + L[f]].astype(int)
    Y, Z = (X + 1) % 3, (X + 2) % 3
    if rho:
        Y, Z = Z, Y
    sy = fac(i, Y) + fac(j, Y)
    sz = fac(j, Z) - s * fac(i, Z)
    vy, vz = bool(np.all(np.abs(sy) <= 1)), bool(np.all(np.abs(sz) <= 1))
    nz = lambda a: int(np.count_nonzero(a))
    f = np.zeros(32)
    f[X] = 1
    f[3] = rho
    f[4] = s < 0
    f[5] = nz(fac(i, X))
    f[6], f[7] = nz(fac(i, Y)), nz(fac(j, Y))
    f[8], f[9] = (nz(sy) if vy else 0), vy
    f[10], f[11] = nz(fac(i, Z)), nz(fac(j, Z))
    f[12], f[13] = (nz(sz) if vz else 0), vz
    f[14] = nz(fac(i, Y) * fac(j, Y))
    f[15] = nz(fac(i, Z) * fac(j, Z))
    f[16] = vy and nz(sy) == 0
    f[17] = vz and nz(sz) == 0
    f[18] = min(k_i, 64)
    f[19] = r - best_r
    f[20] = r
    f[21:24] = fmt
    f[24] = min(q, 64)
    f[31] = 1
    return f


@pytest.mark.parametrize("fmt", FORMATS)
def test_every_feature_equals_its_definition(fmt):
    for scheme, best_r in walked_states(fmt, n=4):
        r = scheme.shape[0]
        i0 = r // 3
        for W in (oracle.WINDOW, 9):
            feat, cand = oracle.window_features(fmt, scheme, best_r, i0, W=W)
            # per-term candidate counts and positions, from the pinned candidate lists
            count = {i: len(candidate_rows(fmt, scheme, i)) for i in range(r)}
            for row, (i, X, j, s, rho) in zip(feat, cand):
                q = (i - i0) % r
                want = features_by_definition(fmt, scheme, r, best_r, i, X, j, s, rho, count[i], q)
                assert np.array_equal(row, want), (fmt, i, X, j, s, rho, row, want)


def unit(L, *pos, neg=()):
    v = np.zeros(L, np.int8)
    for e in pos:
        v[e] = 1
    for e in neg:
        v[e] = -1
    return v


def test_features_on_the_naive_2x2x2_scheme_counted_by_hand():
    """Naive (2,2,2): term (i,k,j) = e_ik (x) e_kj (x) e_ji at row (i*2+k)*2+j.
    Term 0 shares u = e_00 with term 1 (0,0,1), v = e_00 with term 4 (1,0,0) and
    w = e_00 with term 2 (0,1,0): six candidates, in the order (u, 1), (v, 4),
    (w, 2), rho 0 then 1.  Every factor has one non-zero; for (u, term 1):
    Y = v: v_0 + v_1 (two non-zeros, no overlap), Z = w: w_1 - w_0 (two)."""
    fmt = (2, 2, 2)
    scheme = naive_start(*fmt)
    feat, cand = oracle.window_features(fmt, scheme, best_r=8, i0=0, W=6)
    assert [tuple(c) for c in cand] == [(0, 0, 1, 1, 0), (0, 0, 1, 1, 1), (0, 1, 4, 1, 0), (0, 1, 4, 1, 1),
                                       (0, 2, 2, 1, 0), (0, 2, 2, 1, 1)]
    #            X one-hot  rho s  nX nYi nYj nY+ vY nZi nZj nZ- vZ oY oZ 0Y 0Z  ki  r-b  r  m  n  p  q
    want0 = [1, 0, 0, 0, 0, 1, 1, 1, 2, 1, 1, 1, 2, 1, 0, 0, 0, 0, 6, 0, 8, 2, 2, 2, 0]
    assert np.array_equal(feat[0][:25], want0) and np.array_equal(feat[0][25:], [0] * 6 + [1])
    # rho = 1 swaps the roles of v and w: the same counts
    assert np.array_equal(feat[1][:25], [1, 0, 0, 1] + want0[4:])
    # window capacity 6 holds term 0 exactly; from i0 = 7 the first term is 7
    _, cand7 = oracle.window_features(fmt, scheme, best_r=8, i0=7, W=2)
    assert [tuple(c[:1]) for c in cand7] == [(7,), (7,)]


def test_features_of_invalid_and_vanishing_sums_counted_by_hand():
    """A hand-built (2,2,2) state (Eq. (1) is not needed for the features):
    term 0 = (e0, e0 + e1, e2 - e3), term 1 = (e0, -e0 + e1, e2), term 2 = (e1, e2, e3).
    Terms 0 and 1 share u: Y = v gives e0 + e1 - e0 + e1 = 2 e1 (leaves Z_T: invalid),
    Z = w gives w_1 - w_0 = e3 (valid, one non-zero).  With rho = 1 (Y = w,
    Z = v): w_0 + w_1 = 2 e2 - e3 (invalid) and v_1 - v_0 = -2 e0 (invalid)."""
    fmt = (2, 2, 2)
    sch = np.zeros((3, 12), np.int8)
    sch[0] = np.concatenate([unit(4, 0), unit(4, 0, 1), unit(4, 2, neg=(3,))])
    sch[1] = np.concatenate([unit(4, 0), unit(4, 1, neg=(0,)), unit(4, 2)])
    sch[2] = np.concatenate([unit(4, 1), unit(4, 2), unit(4, 3)])
    feat, cand = oracle.window_features(fmt, sch, best_r=2, i0=0, W=2)
    assert [tuple(c) for c in cand] == [(0, 0, 1, 1, 0), (0, 0, 1, 1, 1)]
    #           X      rho s nX nYi nYj nY+ vY nZi nZj nZ- vZ oY oZ 0Y 0Z ki r-b r  m  n  p  q
    want0 = [1, 0, 0, 0, 0, 1, 2, 2, 0, 0, 2, 1, 1, 1, 2, 1, 0, 0, 2, 1, 3, 2, 2, 2, 0]
    want1 = [1, 0, 0, 1, 0, 1, 2, 1, 0, 0, 2, 2, 0, 0, 1, 2, 0, 0, 2, 1, 3, 2, 2, 2, 0]
    assert np.array_equal(feat[0][:25], want0), feat[0][:25]
    assert np.array_equal(feat[1][:25], want1), feat[1][:25]
    # a sum that vanishes: term 1's v replaced by -v_0 on the same support -> Y_i + Y_j = 0
    sch[1, 4:8] = -sch[0, 4:8]
    feat, cand = oracle.window_features(fmt, sch, best_r=3, i0=0, W=1)
    assert feat[0][8] == 0 and feat[0][9] == 1 and feat[0][16] == 1 and feat[0][19] == 0


@pytest.mark.parametrize("fmt,seed", [((3, 3, 3), 3), ((2, 2, 2), 4)])
def test_training_log_is_the_rank_lowering_steps_and_a_philox_sample(fmt, seed):
    """Walk the oracle one window step at a time; before each step compute the
    window of the current state and the uniform choice mulhi(x1, K) from the
    pinned Philox; the log record of the step must be that candidate's features
    with label 1 exactly when the rank fell, and label 0 exactly when it did
    not and Philox(t, walker, sub-stream 256)[0] < the threshold."""
    nw, steps, neg = 6, 150, int(0.3 * 2**32)
    start = naive_start(*fmt)
    ids = np.arange(nw) * 11
    step_by_step = oracle.Walkers(fmt, start, ids, seed=seed, plateau_len=40)
    whole = oracle.Walkers(fmt, start, ids, seed=seed, plateau_len=40).walk_window(steps, threads=2,
                                                                                  log_neg_thresh=neg)
    seen = {0: 0, 1: 0}
    for t in range(steps):
        red_before = step_by_step.info["reductions"].copy()
        states = [(step_by_step.scheme(w), int(step_by_step.info["best_r"][w])) for w in range(nw)]
        step_by_step.walk_window(1, threads=1)
        for w in range(nw):
            scheme, best_r = states[w]
            x = oracle.philox4x32_10([t, 0, int(ids[w]), 0], [seed, 0])
            i0 = (int(x[0]) * scheme.shape[0]) >> 32
            feat, cand = oracle.window_features(fmt, scheme, best_r, i0)
            K = feat.shape[0]
            lab = int(whole.log_label[w, t])
            if K == 0:
                assert lab == -1
                continue
            c = (int(x[1]) * K) >> 32
            # the rank fell at the flip (a later plus transition of the same step may raise it again)
            fell = bool(step_by_step.info["reductions"][w] > red_before[w])
            keep0 = int(oracle.philox4x32_10([t, 0, int(ids[w]), 256], [seed, 0])[0]) < neg
            assert lab == (1 if fell else (0 if keep0 else -1)), (w, t, lab, fell, keep0)
            if lab >= 0:
                seen[lab] += 1
            if lab >= 0:
                assert np.array_equal(whole.log_feat[w, t], feat[c].astype(np.uint8))
    assert int((whole.log_label == 1).sum()) == int(whole.info["reductions"].sum())
    assert seen[1] > 0 and seen[0] > 0
    # the whole walk and the step-by-step walk are the same trajectories
    assert np.array_equal(whole.info["digest"], step_by_step.info["digest"])


def test_horizon_log_by_hand():
    """One walker, nine steps, H = 3: rank-lowering steps 3, 6, 8; sampled
    label-0 steps 1 and 7; step 5 had no candidate.  Step 3 logs the chosen
    steps 1..3, step 6 the chosen steps 4..6 after step 3 (5 had none: 4, 6),
    step 8 the steps 7..8 after 6 (its window 6..8 starts at the previous
    rank-lowering step); steps 1 and 7 also appear with label 0."""
    label = np.array([[-1, 0, -1, 1, -1, -1, 1, 0, 1]], np.int8)
    chosen = np.array([[1, 1, 1, 1, 1, 0, 1, 1, 1]], bool)
    feat = np.zeros((1, 9, 32), np.uint8)
    feat[0, :, 0] = np.arange(9) + 10          # a per-step marker
    wid, st, lab, f = oracle.horizon_log(label, feat, chosen, np.array([42]), 3)
    want = [(1, 0.0), (1, 1.0), (2, 1.0), (3, 1.0), (4, 1.0), (6, 1.0), (7, 0.0), (7, 1.0), (8, 1.0)]
    assert list(zip(st.tolist(), lab.tolist())) == want
    assert (wid == 42).all() and np.array_equal(f[:, 0], st + 10)


@pytest.mark.parametrize("H", [1, 4, 10_000])
def test_horizon_log_on_an_oracle_walk(H):
    """H = 1 is the plain log (the records of label >= 0); any H keeps the
    label-0 records; with H beyond the walk every chosen step up to the last
    rank-lowering step appears once with label 1; label-1 entries never
    exceed H per rank-lowering step."""
    fmt, nw, steps = (3, 3, 3), 8, 400
    start = naive_start(*fmt)
    ids = np.arange(nw) * 5
    o = oracle.Walkers(fmt, start, ids, seed=9, plateau_len=60).walk_window(steps, threads=2,
                                                                            log_neg_thresh=int(0.05 * 2**32))
    wid, st, lab, f = oracle.horizon_log(o.log_label, o.log_feat, o.log_chosen, ids, H)
    zw, zt = np.nonzero(o.log_label == 0)
    assert np.array_equal(np.sort(ids[zw] * steps + zt), np.sort(wid[lab == 0] * steps + st[lab == 0]))
    n_low = int((o.log_label == 1).sum())
    assert n_low > 0
    assert (lab == 1).sum() <= H * n_low
    for k in np.nonzero(lab == 1)[0]:
        w = int(np.nonzero(ids == wid[k])[0][0])
        assert o.log_chosen[w, st[k]]
        assert np.array_equal(f[k], o.log_feat[w, st[k]])
    if H == 1:
        ow, ot = np.nonzero(o.log_label == 1)
        assert np.array_equal(ids[ow] * steps + ot, wid[lab == 1] * steps + st[lab == 1])
    if H >= steps:
        for w in range(nw):
            low = np.nonzero(o.log_label[w] == 1)[0]
            if low.size == 0:
                assert not (wid[lab == 1] == ids[w]).any()
                continue
            want = np.nonzero(o.log_chosen[w, : low[-1] + 1])[0]
            assert np.array_equal(st[(lab == 1) & (wid == ids[w])], want)


def test_adam_first_step_and_constant_gradient_closed_forms():
    """t = 1: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps); with a
    constant gradient the bias corrections keep m_hat = g and v_hat = g^2 on
    every later step, so every update is the same."""
    g = np.array([0.5, -2.0, 1e-3, 0.0, 3.0])
    lr = 0.01
    opt = mlp.Adam(np.zeros(5))
    for k in range(1, 6):
        opt.step(g, lr)
        want = -k * lr * g / (np.abs(g) + 1e-8)
        assert np.allclose(opt.theta, want, rtol=1e-12, atol=1e-15), k


def test_adam_two_steps_by_hand():
    """g = 1 then -1 (beta1 0.9, beta2 0.999): m = 0.1, v = 0.001, then
    m = -0.01, v = 0.001999; m_hat = -0.01 / 0.19, v_hat = 0.001999 / 0.001999 = 1."""
    opt = mlp.Adam(np.zeros(1))
    opt.step(np.array([1.0]), 0.1)
    assert np.isclose(opt.theta[0], -0.1 * 1.0 / (1.0 + 1e-8))
    opt.step(np.array([-1.0]), 0.1)
    m_hat = -0.01 / (1 - 0.9 ** 2)
    assert np.isclose(opt.m[0], -0.01) and np.isclose(opt.v[0], 0.001999)
    assert np.isclose(opt.theta[0], -0.1 / (1.0 + 1e-8) - 0.1 * m_hat / (1.0 + 1e-8), rtol=1e-12)


def test_adam_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    theta0 = rng.normal(size=50)
    grads = [rng.normal(size=50) * 10.0 ** rng.integers(-4, 2) for _ in range(12)]
    opt = mlp.Adam(theta0)
    p = torch.nn.Parameter(torch.tensor(theta0, dtype=torch.float64))
    ref = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    for g in grads:
        opt.step(g, 3e-3)
        p.grad = torch.tensor(g, dtype=torch.float64)
        ref.step()
    assert np.allclose(opt.theta, p.detach().numpy(), rtol=1e-12, atol=1e-14)
