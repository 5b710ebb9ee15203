"""Start schemes for the large formats, built on the host with the library's
meta operators (Section 3.3.2) from verified smaller schemes.  The paper seeds
its searches from published scheme catalogues, which are not available here;
these compositions stand in for them (every result is checked with Eq. (1) by
the library before it is returned)."""
from __future__ import annotations

import numpy as np

from . import tfg
from .workloads import naive_start, strassen_start

AXIS_M, AXIS_N, AXIS_P = 0, 1, 2


def start_223():
    """(2,2,3:11): Strassen extended along p."""
    return tfg.tfg_extend((2, 2, 2), strassen_start(), AXIS_P)


def start_4_5_12():
    """(4,5,12:202) = extend_n(Strassen (x) double_p((2,2,3:11)))."""
    f1, s1 = start_223()
    f2, s2 = tfg.tfg_double(f1, s1, AXIS_P)                  # (2,2,6:22)
    f3, s3 = tfg.tfg_product((2, 2, 2), strassen_start(), f2, s2)   # (4,4,12:154)
    return tfg.tfg_extend(f3, s3, AXIS_N)                     # (4,5,12:202)


def start_6_7_9(scheme_333=None):
    """(6,7,9) = extend_n((2,2,3:11) (x) S333), S333 a verified (3,3,3) scheme
    (the naive rank-27 one by default): rank 11 * r333 + 54."""
    f1, s1 = start_223()
    s333 = naive_start(3, 3, 3) if scheme_333 is None else scheme_333
    f2, s2 = tfg.tfg_product(f1, s1, (3, 3, 3), s333)         # (6,6,9)
    return tfg.tfg_extend(f2, s2, AXIS_N)                     # (6,7,9)


def start_5_6_10():
    """(5,6,10:285) = merge_m(Strassen (x) naive(1,3,5), naive(3,6,10))."""
    fa, sa = tfg.tfg_product((2, 2, 2), strassen_start(), (1, 3, 5), naive_start(1, 3, 5))   # (2,6,10:105)
    return tfg.tfg_merge(fa, sa, (3, 6, 10), naive_start(3, 6, 10), AXIS_M)                  # (5,6,10:285)


def large_populations(walkers: int = 131072, scheme_333=None):
    out = []
    for f, s in [start_4_5_12(), start_5_6_10(), start_6_7_9(scheme_333)]:
        out.append((f, 0, s, walkers))
    return out
