"""Isotropy invariants of a scheme (Section "Isotropy Invariants and Novelty
Verification"), written out from their definitions.

TEST INFRASTRUCTURE ONLY (see the package docstring).

For a scheme (U, V, W) of rank r, term i's factors read as matrices: U_i is
m x n (u[i*n+k] = entry (i, k)), V_i is n x p (v[k*p+j]), W_i is p x m
(w[j*m+i], the C^T convention).  Then

* type polynomial      sum_i X^rank(U_i) Y^rank(V_i) Z^rank(W_i);
* symmetric invariant  the sum of the type polynomial over the six
                       permutations of the variables (x, y, z);
* rank-sum polynomial  w^(sum_i rank U_i) + w^(sum_i rank V_i) + w^(sum_i rank W_i).

Ranks are classical matrix ranks over Q, computed by Gaussian elimination on
exact fractions.  (For Z_2 schemes the same definitions are taken over GF(2):
a reading, the paper computes the invariants of its ternary schemes.)
Polynomials are returned as dicts {exponent tuple: coefficient}.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import permutations

import numpy as np

MODE_ZT, MODE_Z2 = 0, 1


def rank_q(M) -> int:
    """Rank over Q: row reduction with exact fractions."""
    A = [[Fraction(int(x)) for x in row] for row in np.asarray(M)]
    rows = len(A)
    cols = len(A[0]) if rows else 0
    rank = 0
    for c in range(cols):
        piv = next((r for r in range(rank, rows) if A[r][c] != 0), None)
        if piv is None:
            continue
        A[rank], A[piv] = A[piv], A[rank]
        for r in range(rows):
            if r != rank and A[r][c] != 0:
                f = A[r][c] / A[rank][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[rank])]
        rank += 1
    return rank


def rank_gf2(M) -> int:
    """Rank over GF(2): row reduction of the entries mod 2."""
    A = [[int(x) & 1 for x in row] for row in np.asarray(M)]
    rows = len(A)
    cols = len(A[0]) if rows else 0
    rank = 0
    for c in range(cols):
        piv = next((r for r in range(rank, rows) if A[r][c]), None)
        if piv is None:
            continue
        A[rank], A[piv] = A[piv], A[rank]
        for r in range(rows):
            if r != rank and A[r][c]:
                A[r] = [a ^ b for a, b in zip(A[r], A[rank])]
        rank += 1
    return rank


def factor_matrices(fmt, row):
    """The three factors of one term as matrices U (m x n), V (n x p), W (p x m)."""
    m, n, p = fmt
    LU, LV = m * n, n * p
    row = np.asarray(row)
    return (row[:LU].reshape(m, n), row[LU:LU + LV].reshape(n, p), row[LU + LV:].reshape(p, m))


def term_ranks(fmt, scheme, mode=MODE_ZT):
    rk = rank_q if mode == MODE_ZT else rank_gf2
    return [tuple(rk(F) for F in factor_matrices(fmt, row)) for row in np.asarray(scheme)]


def type_polynomial(ranks) -> dict:
    out: dict = {}
    for t in ranks:
        out[t] = out.get(t, 0) + 1
    return out


def symmetric_polynomial(ranks) -> dict:
    out: dict = {}
    for t in ranks:
        for perm in permutations(range(3)):
            e = tuple(t[perm[k]] for k in range(3))
            out[e] = out.get(e, 0) + 1
    return out


def rank_sums(ranks):
    return tuple(sum(t[k] for t in ranks) for k in range(3))


def isotropy_invariants(fmt, scheme, mode=MODE_ZT):
    """(term ranks, type polynomial, symmetric polynomial, rank sums)."""
    tr = term_ranks(fmt, scheme, mode)
    return tr, type_polynomial(tr), symmetric_polynomial(tr), rank_sums(tr)
