"""Pins of the oracle's primitives against values fixed by the paper, by
published test vectors, by textbooks and by brute force."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300.workloads import golden_dir, naive_start, read_scheme

GOLD = golden_dir()


def load(name):
    return read_scheme(os.path.join(GOLD, name))


# Known-answer vectors of Philox4x32-10 published with the Random123 library
# (Salmon et al., SC'11): counter, key -> output.
PHILOX_KAT = [
    ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
    ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
    ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
     [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
]


@pytest.mark.parametrize("ctr,key,want", PHILOX_KAT)
def test_philox_known_answers(ctr, key, want):
    assert list(oracle.philox4x32_10(ctr, key)) == want


def test_paper_example_223_is_valid_in_ct_convention():
    # Section 3.1.1: the printed (2,2,3:11) scheme, columns in the C^T order.
    fmt, s = load("paper_2x2x3_r11.txt")
    assert fmt == (2, 2, 3) and s.shape[0] == 11
    assert oracle.brent_valid(fmt, s)
    # Section 4.5 formula on this scheme: 48 non-zeros - 2*11 - 2*3 = 20.
    assert oracle.additive_complexity(fmt, s) == 20


def test_paper_example_223_is_invalid_in_plain_c_order():
    # Reading W's columns as row-major c_ij (plain C) instead of the C^T order
    # must break Eq. (1): the convention is pinned, not assumed.
    fmt, s = load("paper_2x2x3_r11.txt")
    m, n, p = fmt
    LU, LV = m * n, n * p
    w = s[:, LU + LV:].reshape(-1, p, m)          # stored [j, i]
    s2 = s.copy()
    s2[:, LU + LV:] = np.transpose(w, (0, 2, 1)).reshape(-1, m * p)  # reinterpret as [i, j]
    assert not oracle.brent_valid(fmt, s2)


def test_sign_symmetry_example_exact():
    # Section 3.6: normalising (U, V, W) gives exactly (U', V', W').
    fmt, before = load("paper_sign_example_before.txt")
    _, after = load("paper_sign_example_after.txt")
    assert oracle.brent_valid(fmt, before) and oracle.brent_valid(fmt, after)
    assert np.array_equal(oracle.canonicalize(fmt, before), after)
    # idempotent
    assert np.array_equal(oracle.canonicalize(fmt, after), after)


def test_strassen_valid():
    fmt, s = load("strassen_2x2x2_r7.txt")
    assert oracle.brent_valid(fmt, s)
    assert oracle.brent_valid(fmt, s, oracle.MODE_Z2)


@pytest.mark.parametrize("name", ["strassen_2x2x2_r7.txt", "paper_2x2x3_r11.txt"])
def test_any_single_coefficient_change_is_invalid(name):
    # Changing one coefficient changes the tensor by (delta) * (outer product of
    # the other two non-zero factors), so every such change must be detected.
    fmt, s = load(name)
    for t in range(s.shape[0]):
        for e in range(s.shape[1]):
            for v in (-1, 0, 1):
                if v == s[t, e]:
                    continue
                s2 = s.copy()
                s2[t, e] = v
                assert not oracle.brent_valid(fmt, s2), (t, e, v)


@pytest.mark.parametrize("fmt", [(1, 1, 1), (2, 2, 2), (2, 3, 4), (3, 3, 3), (4, 4, 5), (3, 2, 5)])
def test_naive_scheme_closed_forms(fmt):
    m, n, p = fmt
    s = naive_start(*fmt)
    assert s.shape[0] == m * n * p
    assert oracle.brent_valid(fmt, s) and oracle.brent_valid(fmt, s, oracle.MODE_Z2)
    assert oracle.additive_complexity(fmt, s) == m * p * (n - 1)
    # dropping any one term breaks it
    for t in range(s.shape[0]):
        assert not oracle.brent_valid(fmt, np.delete(s, t, axis=0))


def test_brent_z2_mod_two():
    # 2 = 0 in Z_2: a duplicated term pair cancels mod 2 but not over the integers
    fmt = (2, 2, 2)
    s = naive_start(*fmt)
    extra = np.stack([s[0], s[0]])
    s2 = np.concatenate([s, extra])
    assert oracle.brent_valid(fmt, s2, oracle.MODE_Z2)
    assert not oracle.brent_valid(fmt, s2, oracle.MODE_ZT)


def _tensor(fmt, scheme):
    m, n, p = fmt
    LU, LV = m * n, n * p
    s = scheme.astype(np.int64)
    return np.einsum("la,lb,lc->abc", s[:, :LU], s[:, LU:LU + LV], s[:, LU + LV:])


def _flip_preserves_tensor(fmt, s, i, X, j, sg, rho):
    """Apply the flip formula without any range check and compare tensors."""
    m, n, p = fmt
    lens = [m * n, n * p, p * m]
    offs = [0, lens[0], lens[0] + lens[1]]
    Y, Z = (X + 1) % 3, (X + 2) % 3
    if rho:
        Y, Z = Z, Y
    t = s.astype(np.int64).copy()
    yi = slice(offs[Y], offs[Y] + lens[Y])
    zi = slice(offs[Z], offs[Z] + lens[Z])
    t[i, yi] = s[i, yi].astype(np.int64) + s[j, yi]
    t[j, zi] = s[j, zi].astype(np.int64) - sg * s[i, zi].astype(np.int64)
    return np.array_equal(_tensor(fmt, t), _tensor(fmt, s.astype(np.int64)))


@pytest.mark.parametrize("fmt,seed", [((2, 2, 2), 3), ((2, 2, 3), 4), ((3, 3, 3), 5)])
def test_candidates_equal_brute_force(fmt, seed):
    """The flip candidates of term i are exactly the (X, j, s) whose flip leaves
    the tensor unchanged, in the order (X, j, rho)."""
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(4), seed=seed, plateau_len=300)
    for _ in range(6):
        W.walk(400)
        for w in range(4):
            s = W.scheme(w)
            r = s.shape[0]
            for i in range(r):
                got = [tuple(x) for x in oracle.enumerate_candidates(fmt, s, i)]
                want = []
                for X in range(3):
                    for j in range(r):
                        if j == i:
                            continue
                        for sg in (1, -1):
                            if _flip_preserves_tensor(fmt, s, i, X, j, sg, 0):
                                assert _flip_preserves_tensor(fmt, s, i, X, j, sg, 1)
                                want += [(X, j, sg, 0), (X, j, sg, 1)]
                assert got == want


def test_ternary_addition_truth_table():
    """Section 3.5.2: addition/subtraction of ternary vectors is valid exactly
    when no position would reach +-2; checked on all pairs of length-3 vectors
    through the flip, whose two sums are Y_i + Y_j and Z_j - s Z_i."""
    vals = list(itertools.product((-1, 0, 1), repeat=3))
    # a (1,1,3) scheme gives factor lengths 1, 3, 3: use V as the summed factor.
    fmt = (1, 1, 3)
    for a in vals:
        if not any(a):
            continue
        for b in vals:
            if not any(b):
                continue
            # two terms sharing u = (1); flip X=U, rho=0: V_0 += V_1, W_1 -= W_0
            s = np.zeros((2, 7), np.int8)
            s[:, 0] = 1
            s[0, 1:4] = a
            s[1, 1:4] = b
            s[0, 4:7] = (1, 0, 0)
            s[1, 4:7] = (0, 1, 0)
            action, _ = oracle.apply_flip(fmt, s, 0, 0, 1, 1, 0)
            want_valid = all(abs(x + y) <= 1 for x, y in zip(a, b))
            assert action == (oracle.ACCEPT if want_valid else oracle.REJECT), (a, b)
