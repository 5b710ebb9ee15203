"""Pins of the oracle walker: invariants after every step, brute-force
reachability, best-scheme bookkeeping, determinism and resume."""
import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300.workloads import golden_dir, naive_start, read_scheme
import os


@pytest.mark.parametrize("mode", [oracle.MODE_ZT, oracle.MODE_Z2])
@pytest.mark.parametrize("fmt,L,steps", [((2, 2, 2), 150, 6000), ((2, 2, 3), 300, 4000),
                                         ((3, 3, 3), 800, 3000), ((2, 3, 4), 400, 3000)])
def test_invariants_after_every_step(fmt, L, steps, mode):
    """Debug mode re-checks after every step: Eq. (1) holds, every term is in
    sign-normal form (Z_T), no factor is zero, and no two terms are reducible."""
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(6), seed=11, mode=mode,
                       plateau_len=L, debug_checks=True)
    W.walk(steps)
    info = W.info
    assert (info["debug_failures"] == 0).all()
    assert (info["t"] == steps).all()
    assert (info["plus"] > 0).any(), "plateau length chosen so that plus transitions happen"
    assert (info["merges"] > 0).any()
    assert (info["accepted"] + info["rejected"] + info["nocand"] == steps).all()
    if mode == oracle.MODE_Z2:
        assert (info["rejected"] == 0).all()
    for w in range(6):
        assert oracle.brent_valid(fmt, W.best_scheme(w), mode)
        assert W.info["best_r"][w] <= W.info["r"][w]
        assert W.info["r"][w] <= W.info["best_r"][w] + 3
        assert W.info["r"][w] <= W.r_max


def test_bfs_depth3_from_naive_222():
    """Every state reachable in <= 3 flips from the naive (2,2,2) scheme (all
    sampled terms, all candidates) satisfies Eq. (1) and sign normalisation."""
    fmt = (2, 2, 2)
    start = oracle.prepare_start(fmt, naive_start(*fmt))
    frontier = {start.tobytes(): start}
    seen = set(frontier)
    n_states = 0
    for depth in range(3):
        nxt = {}
        for s in frontier.values():
            for i in range(s.shape[0]):
                for (X, j, sg, rho) in oracle.enumerate_candidates(fmt, s, i):
                    action, s2 = oracle.apply_flip(fmt, s, i, X, j, sg, rho)
                    if action != oracle.ACCEPT:
                        continue
                    key = s2.tobytes() + bytes([s2.shape[0]])
                    if key in seen:
                        continue
                    seen.add(key)
                    assert oracle.brent_valid(fmt, s2)
                    assert np.array_equal(oracle.canonicalize(fmt, s2), s2)
                    nxt[key] = s2
                    n_states += 1
        frontier = nxt
    assert n_states > 100


def test_best_tracks_running_minimum():
    """best_r is the running minimum of r; best_t is the step where it last fell."""
    fmt = (2, 2, 2)
    W = oracle.Walkers(fmt, naive_start(*fmt), [5], seed=2, plateau_len=100)
    run_min, last_fall = W.info["r"][0], 0
    for t in range(3000):
        W.walk(1, threads=1)
        r = W.info["r"][0]
        if r < run_min:
            run_min, last_fall = r, t
        assert W.info["best_r"][0] == run_min
        if run_min < W.r0:
            assert W.info["best_t"][0] == last_fall


def test_deterministic_and_thread_independent():
    fmt = (3, 3, 3)
    a = oracle.Walkers(fmt, naive_start(*fmt), np.arange(12), seed=7, plateau_len=500).walk(3000, threads=1)
    b = oracle.Walkers(fmt, naive_start(*fmt), np.arange(12), seed=7, plateau_len=500).walk(3000, threads=5)
    assert np.array_equal(a.slots, b.slots) and np.array_equal(a.best, b.best)
    assert np.array_equal(a.info, b.info)
    c = oracle.Walkers(fmt, naive_start(*fmt), np.arange(12), seed=8, plateau_len=500).walk(3000)
    assert not np.array_equal(a.info["digest"], c.info["digest"])


def test_resume_equals_uninterrupted():
    fmt = (2, 2, 3)
    a = oracle.Walkers(fmt, naive_start(*fmt), np.arange(8), seed=1, plateau_len=200).walk(2000)
    b = oracle.Walkers(fmt, naive_start(*fmt), np.arange(8), seed=1, plateau_len=200)
    b.walk(700).walk(1300)
    assert np.array_equal(a.slots, b.slots) and np.array_equal(a.info, b.info)


def test_walker_ids_select_streams():
    """A walker's trajectory depends only on (seed, walker id, step): walker 9
    alone equals walker 9 inside a batch."""
    fmt = (2, 2, 2)
    batch = oracle.Walkers(fmt, naive_start(*fmt), np.arange(16), seed=3, plateau_len=100).walk(2000)
    solo = oracle.Walkers(fmt, naive_start(*fmt), [9], seed=3, plateau_len=100).walk(2000)
    assert np.array_equal(batch.slots[9], solo.slots[0])
    assert batch.info[9] == solo.info[0]


def test_prepare_start_reduces_duplicates():
    """A scheme with a duplicated term pair (shared u, v) merges on preparation;
    the Strassen scheme, which has no reducible pair, is left at rank 7."""
    fmt, s = read_scheme(os.path.join(golden_dir(), "strassen_2x2x2_r7.txt"))
    p = oracle.prepare_start(fmt, s)
    assert p.shape[0] == 7 and oracle.brent_valid(fmt, p)
    # split term 0 into two halves sharing u and v: w = w1 + w2
    s2 = np.concatenate([s, s[:1]])
    s2[0, 8:] = [1, 0, 0, 0]
    s2[7, 8:] = [0, 0, 0, 1]
    assert oracle.brent_valid(fmt, s2)
    p2 = oracle.prepare_start(fmt, s2)
    assert p2.shape[0] == 7 and oracle.brent_valid(fmt, p2)


def test_reaches_rank7_from_naive_z2():
    """The flip-graph literature the paper builds on (Section 2.2.4) walks the
    naive 2x2x2 scheme down to rank 7; over Z_2 every walker gets there fast."""
    fmt = (2, 2, 2)
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(32), seed=0, mode=oracle.MODE_Z2,
                       plateau_len=1000).walk(20000)
    assert (W.info["best_r"] == 7).all()


@pytest.mark.parametrize("mode", [oracle.MODE_ZT, oracle.MODE_Z2])
@pytest.mark.parametrize("fmt", [(2, 2, 2), (2, 3, 3), (3, 3, 3)])
def test_algorithm1_policy_invariants(fmt, mode):
    """Walk policy 1 (Algorithm 1: expand after a failed try_flip and with
    probability p_expand; expand = plus or split): Eq. (1), normal form, no zero
    factor and no reducible pair after every step; expansions happen, the rank
    never exceeds the capacity, and the best rank is the running minimum."""
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(6), seed=21, mode=mode, r_slack=10, policy=1,
                       expand_thresh=int(0.03 * 2**32), debug_checks=True)
    best_seen = np.full(6, W.r0)
    for _ in range(10):
        W.walk(300)
        best_seen = np.minimum(best_seen, W.info["r"])
        assert (W.info["best_r"] <= best_seen).all()
    info = W.info
    assert (info["debug_failures"] == 0).all()
    assert (info["plus"] > 0).all()
    assert (info["r"] <= W.r_max).all() and (info["r"] > 0).all()
    for w in range(6):
        assert oracle.brent_valid(fmt, W.best_scheme(w), mode) and oracle.brent_valid(fmt, W.scheme(w), mode)


def test_policy0_unaffected_by_expand_threshold():
    """The p_expand threshold and the split operator exist only under policy 1."""
    fmt = (2, 3, 3)
    A = oracle.Walkers(fmt, naive_start(*fmt), np.arange(4), seed=5, plateau_len=200).walk(3000)
    B = oracle.Walkers(fmt, naive_start(*fmt), np.arange(4), seed=5, plateau_len=200,
                       expand_thresh=2**31).walk(3000)
    assert np.array_equal(A.info, B.info) and np.array_equal(A.slots, B.slots)


@pytest.mark.parametrize("mode", [oracle.MODE_ZT, oracle.MODE_Z2])
@pytest.mark.parametrize("fmt", [(2, 2, 3), (3, 3, 3), (2, 3, 4)])
def test_complexity_policy(fmt, mode):
    """Walk policy 2 (naive additive complexity minimisation): flips and zero-term
    removal only -- no merges, no expansions -- Eq. (1), normal form and no zero
    factor after every step; best_nnz is the non-zero count of the best scheme and
    the best (rank, non-zeros) pair is the running minimum."""
    src = oracle.Walkers(fmt, naive_start(*fmt), np.arange(1), seed=3, mode=mode, plateau_len=300).walk(3000)
    start = src.scheme(0)                       # a walked state: more non-zeros than needed
    W = oracle.Walkers(fmt, start, np.arange(6), seed=8, mode=mode, policy=2, debug_checks=True)
    key = [(int(W.info["best_r"][w]), int(W.info["best_nnz"][w])) for w in range(6)]
    assert key[0][1] == int((W.start != 0).sum())
    for _ in range(8):
        W.walk(400)
        for w in range(6):
            now = (int(W.info["best_r"][w]), int(W.info["best_nnz"][w]))
            assert now <= key[w]
            key[w] = now
            b = W.best_scheme(w)
            assert int((b != 0).sum()) == now[1] and oracle.brent_valid(fmt, b, mode)
    info = W.info
    assert (info["debug_failures"] == 0).all()
    assert (info["merges"] == 0).all() and (info["plus"] == 0).all()
    assert any(k[1] < int((W.start != 0).sum()) for k in key), "some walker lowers the non-zero count"
