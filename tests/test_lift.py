"""Z_2 -> Z_T sign lifting (tfg_lift_signs) against independent checks: schemes
known to lift (the sign-stripped Z_T schemes), the oracle's exhaustive
enumeration and backtracking (both exhaustive, neither uses the library's
linear algebra), Eq. (1) on every result, and input validation."""
import os

import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300 import tfg
from paper_2511_20317_gb300.workloads import golden_dir, naive_start, read_scheme, strassen_start


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_20317_gb300 import _build
    _build.build()
    tfg.lib()


def _check_lift(fmt, z2, out):
    assert np.array_equal(np.abs(out), np.abs(z2).astype(np.int8))
    assert oracle.brent_valid(fmt, out, oracle.MODE_ZT)
    assert np.array_equal(oracle.canonicalize(fmt, out), out)


def test_sign_stripped_ternary_schemes_lift():
    cases = [((2, 2, 2), strassen_start()), read_scheme(os.path.join(golden_dir(), "paper_2x2x3_r11.txt"))]
    for fmt, seed in [((2, 3, 4), 1), ((3, 3, 3), 2), ((4, 4, 4), 3)]:
        W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(4), seed=seed, plateau_len=500).walk(4000)
        cases += [(fmt, W.scheme(w)) for w in range(4)]
    for fmt, s in cases:
        z2 = np.abs(s).astype(np.int8)
        out, nodes = tfg.tfg_lift_signs(fmt, z2)
        _check_lift(fmt, z2, out)


@pytest.mark.parametrize("fmt", [(2, 2, 2), (1, 2, 3), (2, 1, 3), (1, 3, 2)])
def test_lift_agrees_with_exhaustive_enumeration(fmt):
    """Small Z_2 schemes with at most 22 free signs: every assignment is tried."""
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(60), seed=7, mode=oracle.MODE_Z2, plateau_len=300).walk(3000)
    decided = 0
    for w in range(60):
        for s in (W.best_scheme(w), W.scheme(w)):
            bf = oracle.lift_bruteforce(fmt, s, max_bits=22)
            if bf is None:
                continue
            decided += 1
            try:
                out, _ = tfg.tfg_lift_signs(fmt, s)
                ok = True
            except tfg.TfgError as e:
                assert e.code == tfg.TFG_ESCHEME
                ok = False
            assert ok == bf[0]
            if ok:
                _check_lift(fmt, s, out)
    assert decided >= 10


def test_lift_agrees_with_backtracking_including_non_liftable():
    seen = {True: 0, False: 0}
    for fmt, walkers in [((1, 2, 4), 120), ((2, 2, 4), 24)]:
        W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(walkers), seed=11, mode=oracle.MODE_Z2, plateau_len=50,
                           r_slack=6).walk(400)
        for w in range(walkers):
            s = W.scheme(w)
            bt = oracle.lift_backtrack(fmt, s, max_nodes=200_000)
            if bt is None:
                continue
            try:
                out, _ = tfg.tfg_lift_signs(fmt, s)
                ok = True
            except tfg.TfgError as e:
                assert e.code == tfg.TFG_ESCHEME
                ok = False
            assert ok == bt[0], (fmt, w)
            seen[ok] += 1
            if ok:
                _check_lift(fmt, s, out)
    assert seen[True] > 50 and seen[False] >= 2


def test_z2_rank23_333_schemes_lift_to_ternary():
    """Z_2 walks reach (3,3,3) rank 23; some of those schemes lift to Z_T rank 23."""
    fmt = (3, 3, 3)
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(16), seed=1, mode=oracle.MODE_Z2,
                       plateau_len=50000).walk(200000)
    lifted = 0
    for w in np.flatnonzero(W.info["best_r"] == 23):
        s = W.best_scheme(int(w))
        try:
            out, _ = tfg.tfg_lift_signs(fmt, s, max_nodes=10**6)
        except tfg.TfgError:
            continue
        _check_lift(fmt, s, out)
        assert tfg.tfg_verify(fmt, out) and out.shape[0] == 23
        lifted += 1
    assert lifted >= 1


def test_lift_rejects_bad_input():
    z2 = np.abs(strassen_start()).astype(np.int8)
    bad = z2.copy()
    bad[0, 0] = -1
    with pytest.raises(tfg.TfgError) as e:
        tfg.tfg_lift_signs((2, 2, 2), bad)
    assert e.value.code == tfg.TFG_EINVAL
    bad = z2.copy()
    bad[0, 1] ^= 1                                     # Eq. (1) fails mod 2
    with pytest.raises(tfg.TfgError) as e:
        tfg.tfg_lift_signs((2, 2, 2), bad)
    assert e.value.code == tfg.TFG_EINVAL
