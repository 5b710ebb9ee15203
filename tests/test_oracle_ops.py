"""The oracle's instrumented algorithmic op count (the numerator of the walk
kernels' roofline), pinned against its definition recomputed from what each
step visibly did: walking one step at a time, the rank before the step and
which counter the step advanced (no candidate, rejected, accepted) give the
step's operations; the accumulated count must equal their sum."""
import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300.workloads import naive_start

SEARCH = {0: 8, 1: 3}     # word tests per other slot: Z_T u, v exact (2 each), w either sign (4); Z_2 3
FLIP = {0: 18, 1: 2}      # the two new factors: Z_T validity 3 + result 6 each; Z_2 one XOR each
PHILOX = 100              # 10 rounds of 10 operations


@pytest.mark.parametrize("fmt,mode", [((2, 2, 2), 0), ((3, 3, 3), 0), ((3, 3, 3), 1), ((2, 3, 4), 0)])
def test_op_count_is_the_sum_of_each_steps_operations(fmt, mode):
    nw, steps = 5, 300
    w = oracle.Walkers(fmt, naive_start(*fmt), np.arange(nw) * 3, seed=2, mode=mode, plateau_len=40)
    want = np.zeros(nw, np.int64)
    for _ in range(steps):
        r0 = w.info["r"].astype(np.int64).copy()
        acc0, rej0, noc0 = (w.info[k].copy() for k in ("accepted", "rejected", "nocand"))
        w.walk(1, 1)
        acc = w.info["accepted"] - acc0
        rej = w.info["rejected"] - rej0
        noc = w.info["nocand"] - noc0
        assert (acc + rej + noc == 1).all()
        search = SEARCH[mode] * (r0 - 1)
        want += PHILOX + search + (acc + rej) * FLIP[mode] + acc * 2 * search
    assert np.array_equal(w.info["ops"], want)


def test_op_count_by_hand_on_one_step():
    """On the naive (2,2,2) scheme every term shares each of its factors (unit
    matrices) with exactly one other term, and the sum or difference of two
    distinct unit matrices stays in Z_T, so the first step of every walker
    flips: the draw 100, the search over the seven other slots 8 * 7, the two
    new factors 18 and the reduction check of both 2 * 8 * 7: 286."""
    w = oracle.Walkers((2, 2, 2), naive_start(2, 2, 2), np.arange(3), seed=0, plateau_len=10**6)
    w.walk(1, 1)
    assert (w.info["accepted"] == 1).all()
    assert (w.info["ops"] == 286).all()
