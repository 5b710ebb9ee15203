"""Pins of the oracle's isotropy invariants: matrix ranks against brute force,
closed forms (naive scheme, Strassen's scheme), and invariance under the
isotropies of the matrix-multiplication tensor and its cyclic symmetry."""
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import invariants as inv
from paper_2511_20317_gb300.workloads import golden_dir, naive_start, read_scheme


def _det(M):
    """Integer determinant by the Leibniz formula (brute force)."""
    n = len(M)
    tot = 0
    for perm in itertools.permutations(range(n)):
        sign = 1
        for a in range(n):
            for b in range(a + 1, n):
                if perm[a] > perm[b]:
                    sign = -sign
        prod = 1
        for a in range(n):
            prod *= int(M[a][perm[a]])
        tot += sign * prod
    return tot


def _rank_by_minors(M):
    M = np.asarray(M)
    rows, cols = M.shape
    for k in range(min(rows, cols), 0, -1):
        for rs in itertools.combinations(range(rows), k):
            for cs in itertools.combinations(range(cols), k):
                if _det(M[np.ix_(rs, cs)]) != 0:
                    return k
    return 0


def _rank_gf2_by_span(M):
    """log2 of the number of distinct GF(2) combinations of the rows."""
    M = np.asarray(M) & 1
    span = set()
    for mask in range(1 << M.shape[0]):
        v = np.zeros(M.shape[1], dtype=np.int64)
        for a in range(M.shape[0]):
            if (mask >> a) & 1:
                v ^= M[a]
        span.add(v.tobytes())
    return int(np.log2(len(span)))


def test_rank_q_equals_largest_nonzero_minor():
    rng = np.random.default_rng(0)
    for _ in range(300):
        rows, cols = rng.integers(1, 5), rng.integers(1, 6)
        M = rng.integers(-2, 3, size=(rows, cols))
        if rng.random() < 0.3:   # force dependent rows
            M[-1] = M[0] * rng.integers(-2, 3)
        assert inv.rank_q(M) == _rank_by_minors(M), M


def test_rank_gf2_equals_span_size():
    rng = np.random.default_rng(1)
    for _ in range(300):
        rows, cols = rng.integers(1, 6), rng.integers(1, 7)
        M = rng.integers(0, 2, size=(rows, cols))
        assert inv.rank_gf2(M) == _rank_gf2_by_span(M), M


@pytest.mark.parametrize("fmt", [(2, 2, 2), (2, 3, 4), (3, 3, 3), (4, 5, 3)])
def test_naive_scheme_closed_form(fmt):
    r = fmt[0] * fmt[1] * fmt[2]
    tr, typ, sym, sums = inv.isotropy_invariants(fmt, naive_start(*fmt))
    assert tr == [(1, 1, 1)] * r
    assert typ == {(1, 1, 1): r} and sym == {(1, 1, 1): 6 * r} and sums == (r, r, r)


def test_strassen_type_invariant():
    """Strassen's products: M1 = (A11 + A22)(B11 + B22) enters C11 and C22, so all
    three of its factors are rank 2; each of M2..M7 has one factor that is a single
    entry or a sum/difference within one row or column, every factor rank 1:
    type polynomial X^2 Y^2 Z^2 + 6 XYZ."""
    fmt, S = read_scheme(os.path.join(golden_dir(), "strassen_2x2x2_r7.txt"))
    tr, typ, sym, sums = inv.isotropy_invariants(fmt, S)
    assert typ == {(2, 2, 2): 1, (1, 1, 1): 6}
    assert sym == {(2, 2, 2): 6, (1, 1, 1): 36}
    assert sums == (8, 8, 8)


def _signed_perm(n, rng):
    P = np.zeros((n, n), dtype=np.int64)
    P[np.arange(n), rng.permutation(n)] = rng.choice([-1, 1], size=n)
    return P


def _isotropy(fmt, scheme, P, Q, R):
    """Terms (U, V, W) -> (P U Q^-1, Q V R^-1, R W P^-1): tr(ABC) is unchanged."""
    m, n, p = fmt
    rows = []
    for row in np.asarray(scheme):
        U, V, W = inv.factor_matrices(fmt, row)
        U2 = P @ U @ np.linalg.inv(Q).round().astype(np.int64)
        V2 = Q @ V @ np.linalg.inv(R).round().astype(np.int64)
        W2 = R @ W @ np.linalg.inv(P).round().astype(np.int64)
        rows.append(np.concatenate([U2.reshape(-1), V2.reshape(-1), W2.reshape(-1)]))
    return np.array(rows, dtype=np.int8)


@pytest.mark.parametrize("fmt", [(2, 2, 3), (3, 3, 3), (2, 3, 4)])
def test_invariants_unchanged_by_isotropies(fmt):
    rng = np.random.default_rng(7)
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(4), seed=3, plateau_len=300).walk(3000)
    for w in range(4):
        s = W.best_scheme(w)
        base = inv.isotropy_invariants(fmt, s)
        for _ in range(3):
            P, Q, R = _signed_perm(fmt[0], rng), _signed_perm(fmt[1], rng), _signed_perm(fmt[2], rng)
            s2 = _isotropy(fmt, s, P, Q, R)
            assert oracle.brent_valid(fmt, s2)
            assert inv.isotropy_invariants(fmt, s2) == base


def test_cyclic_symmetry_rotates_type_and_keeps_symmetric_invariant():
    fmt, s = read_scheme(os.path.join(golden_dir(), "paper_2x2x3_r11.txt"))
    tr, typ, sym, sums = inv.isotropy_invariants(fmt, s)
    f2, s2 = oracle.cyclic(fmt, s)
    tr2, typ2, sym2, sums2 = inv.isotropy_invariants(f2, s2)
    assert sorted(tr2) == sorted((b, c, a) for a, b, c in tr) or sorted(tr2) == sorted((c, a, b) for a, b, c in tr)
    assert sym2 == sym and sorted(sums2) == sorted(sums)
