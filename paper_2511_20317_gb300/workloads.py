"""Synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the method: it only builds start schemes
(the naive rank-mnp scheme), reads scheme text files, and describes the
walker populations of the measured workloads.  The paper searches from
external scheme catalogues (Section 3.8), which are not available here; the
naive schemes and host-built meta-operator starts stand in for them.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np


def naive_start(m: int, n: int, p: int) -> np.ndarray:
    """Rank-mnp start: term (i,k,j) is a_ik * b_kj -> c_ij (unit vectors), in the
    row layout u[i*n+k] | v[k*p+j] | w[j*m+i]."""
    LU, LV, LW = m * n, n * p, p * m
    out = np.zeros((m * n * p, LU + LV + LW), dtype=np.int8)
    t = 0
    for i in range(m):
        for k in range(n):
            for j in range(p):
                out[t, i * n + k] = 1
                out[t, LU + k * p + j] = 1
                out[t, LU + LV + j * m + i] = 1
                t += 1
    return out


def strassen_start() -> np.ndarray:
    """Strassen's rank-7 (2,2,2) scheme (Numer. Math. 13, 1969), textbook products
    M1..M7 in the row layout u | v | w (w in the C^T order c11 c21 c12 c22)."""
    U = [[1, 0, 0, 1], [0, 0, 1, 1], [1, 0, 0, 0], [0, 0, 0, 1], [1, 1, 0, 0], [-1, 0, 1, 0], [0, 1, 0, -1]]
    V = [[1, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, -1], [-1, 0, 1, 0], [0, 0, 0, 1], [1, 1, 0, 0], [0, 0, 1, 1]]
    W = [[1, 0, 0, 1], [0, 1, 0, -1], [0, 0, 1, 1], [1, 1, 0, 0], [-1, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0]]
    return np.concatenate([np.array(U), np.array(V), np.array(W)], axis=1).astype(np.int8)


def read_scheme(path: str):
    """Parse the text format of tests/golden: 'format m n p', 'rank r', then the
    U, V and W blocks (one row per term).  Returns ((m,n,p), int8 [r, LT])."""
    fmt = rank = None
    blocks: dict[str, list[list[int]]] = {}
    cur = None
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("format"):
                fmt = tuple(int(x) for x in line.split()[1:4])
            elif line.startswith("rank"):
                rank = int(line.split()[1])
            elif line in ("U", "V", "W"):
                cur = line
                blocks[cur] = []
            else:
                blocks[cur].append([int(x) for x in line.split()])
    U, V, W = (np.array(blocks[k], dtype=np.int8) for k in "UVW")
    assert U.shape[0] == V.shape[0] == W.shape[0] == rank
    return fmt, np.concatenate([U, V, W], axis=1)


def largest_remainder_split(total: int, ratios) -> list[int]:
    """Split `total` walkers in proportion to `ratios`, rounding by largest remainder
    (ties to the earlier entry)."""
    s = sum(ratios)
    exact = [total * r / s for r in ratios]
    base = [int(np.floor(e)) for e in exact]
    rem = total - sum(base)
    order = sorted(range(len(ratios)), key=lambda a: (-(exact[a] - base[a]), a))
    for a in order[:rem]:
        base[a] += 1
    return base


@dataclass
class Population:
    """One format's share of a walker population."""
    fmt: tuple
    walkers: int
    mode: int = 0              # 0: Z_T, 1: Z_2
    start: np.ndarray | None = None

    def start_scheme(self) -> np.ndarray:
        return self.start if self.start is not None else naive_start(*self.fmt)


@dataclass
class Workload:
    name: str
    populations: list
    steps: int                 # steps per walker of the full workload
    plateau: int
    seed: int = 0
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def total_walkers(self) -> int:
        return sum(p.walkers for p in self.populations)


def workload_222() -> Workload:
    """(2,2,2) Z_T from the naive rank-8 scheme, 1024 walkers, 1e5 steps, plateau 1e4."""
    return Workload("2x2x2-ZT-naive8-1024w", [Population((2, 2, 2), 1024)], 100_000, 10_000)


def workload_333(mode: int = 0) -> Workload:
    """(3,3,3) from the naive rank-27 scheme, 65536 walkers, 1e6 steps, plateau 5e4.
    Seed 0 for Z_T, seed 1 for Z_2."""
    tag = "ZT" if mode == 0 else "Z2"
    return Workload(f"3x3x3-{tag}-naive27-65536w", [Population((3, 3, 3), 65536, mode)],
                    1_000_000, 50_000, seed=mode)


MIXED_FORMATS = [(2, 4, 5), (3, 3, 4), (3, 4, 5), (4, 4, 4), (4, 4, 5)]
MIXED_RATIOS = [1, 2, 2, 4, 4]


def workload_mixed(total: int = 262144) -> Workload:
    """Five formats in ratios 1:2:2:4:4 of `total` walkers, naive starts, Z_T."""
    split = largest_remainder_split(total, MIXED_RATIOS)
    pops = [Population(f, w) for f, w in zip(MIXED_FORMATS, split)]
    return Workload(f"mixed5-ZT-naive-{total}w", pops, 1_000_000, 50_000)


def golden_dir() -> str:
    return os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")
