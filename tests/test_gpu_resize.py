"""Device resize (tfg_resize) against the oracle's meta operators: every
operator, both modes, per-walker schemes of different ranks; the resized
walkers then walk on and are replayed by oracle walkers started from the
oracle's results."""
import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300 import tfg
from paper_2511_20317_gb300.workloads import naive_start

pytestmark = pytest.mark.gpu

THREADS = 8
SRC = (2, 2, 3)
NW = 24


def _oracle_op(op, fmt, s, axis, index, aux, mode):
    if op == tfg.TFG_RESIZE_PROJECT:
        return oracle.project(fmt, s, axis, index, mode)
    if op == tfg.TFG_RESIZE_EXTEND:
        return oracle.extend(fmt, s, axis, mode)
    if op == tfg.TFG_RESIZE_DOUBLE:
        return oracle.double(fmt, s, axis, mode)
    if op == tfg.TFG_RESIZE_MERGE:
        return oracle.merge(fmt, s, aux[0], aux[1], axis, mode)
    if op == tfg.TFG_RESIZE_PRODUCT:
        return oracle.product(fmt, s, aux[0], aux[1], mode)
    return oracle.swap_sizes(fmt, s, index, mode)


def _mode_rows(s, mode):
    return np.abs(s).astype(np.int8) if mode == tfg.TFG_MODE_Z2 else np.asarray(s, np.int8)


CASES = [
    (tfg.TFG_RESIZE_PROJECT, 0, 1, None),
    (tfg.TFG_RESIZE_PROJECT, 1, 0, None),
    (tfg.TFG_RESIZE_PROJECT, 2, 2, None),
    (tfg.TFG_RESIZE_EXTEND, 0, 0, None),
    (tfg.TFG_RESIZE_EXTEND, 1, 0, None),
    (tfg.TFG_RESIZE_EXTEND, 2, 0, None),
    (tfg.TFG_RESIZE_DOUBLE, 0, 0, None),
    (tfg.TFG_RESIZE_DOUBLE, 2, 0, None),
    (tfg.TFG_RESIZE_MERGE, 2, 0, (2, 2, 1)),
    (tfg.TFG_RESIZE_MERGE, 0, 0, (1, 2, 3)),
    (tfg.TFG_RESIZE_PRODUCT, 0, 0, (1, 2, 1)),
    (tfg.TFG_RESIZE_SWAP, 0, 1, None),
    (tfg.TFG_RESIZE_SWAP, 0, 2, None),
    (tfg.TFG_RESIZE_SWAP, 0, 3, None),
    (tfg.TFG_RESIZE_SWAP, 0, 4, None),
    (tfg.TFG_RESIZE_SWAP, 0, 5, None),
]


@pytest.mark.parametrize("mode", [tfg.TFG_MODE_ZT, tfg.TFG_MODE_Z2])
@pytest.mark.parametrize("op,axis,index,aux_fmt", CASES)
def test_device_resize_matches_oracle_and_walks_on(op, axis, index, aux_fmt, mode):
    # source schemes: oracle walkers of (2,2,3) after a few hundred steps (ranks differ)
    src_start = _mode_rows(naive_start(*SRC), mode)
    gen = oracle.Walkers(SRC, src_start, np.arange(NW), seed=5, mode=mode, plateau_len=80).walk(400, THREADS)
    aux = None
    if aux_fmt is not None:
        aux = (aux_fmt, _mode_rows(naive_start(*aux_fmt), mode))
    out_fmt, _ = _oracle_op(op, SRC, src_start, axis, index, aux, mode)
    slack = 16
    pops = [(SRC, mode, src_start, NW), (out_fmt, mode, _mode_rows(naive_start(*out_fmt), mode), NW)]
    W = tfg.Walkers(pops, seed=11, params=tfg.tfg_default_params(plateau_len=120, r_slack=slack))
    for w in range(NW):
        W.reseed(w, 1, gen.scheme(w))
    info_s, slots_s, _ = W.read_walkers(0, NW)
    first = W.pop[1]["first"]
    skipped = W.resize(op, 0, first, NW, axis=axis, index=index, aux=aux)
    assert skipped == 0
    info, slots, best = W.read_walkers(first, NW)
    R = W.pop[1]["r_max"]
    results = []
    for w in range(NW):
        src = slots_s[w, : info_s["r"][w]]
        f2, want = _oracle_op(op, SRC, src, axis, index, aux, mode)
        assert f2 == out_fmt
        r = want.shape[0]
        assert info["r"][w] == r and info["best_r"][w] == r, (w, info["r"][w], r)
        assert np.array_equal(slots[w, :r], want), f"walker {w}: resized scheme differs"
        assert np.array_equal(best[w, :r], want)
        assert info["plateau"][w] == 0 and info["t"][w] == 0
        assert info["best_nnz"][w] == np.count_nonzero(want)
        assert oracle.brent_valid(out_fmt, want, mode)
        results.append(want)
    assert W.verify_all() == 0
    # the resized walkers walk on exactly like oracle walkers started from the oracle's results
    W.walk(300)
    info, slots, best = W.read_walkers(first, NW)
    for w in range(NW):
        r0 = results[w].shape[0]
        ref = oracle.Walkers(out_fmt, results[w], [first + w], seed=11, mode=mode, plateau_len=120,
                             r_slack=R - r0, prepared=True).walk(300, 1)
        for f in ("r", "best_r", "t", "digest", "accepted", "rejected", "merges", "plus"):
            assert info[f][w] == ref.info[f][0], (w, f, info[f][w], ref.info[f][0])
        assert np.array_equal(slots[w, : info["r"][w]], ref.slots[0, : ref.info["r"][0]])
    W.close()


def test_device_resize_from_best_and_errors():
    mode = tfg.TFG_MODE_ZT
    src_start = naive_start(*SRC)
    pops = [(SRC, mode, src_start, NW), ((2, 2, 4), mode, naive_start(2, 2, 4), NW),
            ((2, 4, 3), mode, naive_start(2, 4, 3), 4)]
    W = tfg.Walkers(pops, seed=3, params=tfg.tfg_default_params(plateau_len=60, r_slack=3))
    W.walk(500)
    info_s, _, best_s = W.read_walkers(0, NW)
    f1 = W.pop[1]["first"]
    # from the best schemes
    assert W.resize(tfg.TFG_RESIZE_EXTEND, 0, f1, NW, axis=2, use_best=True) == 0
    info, slots, _ = W.read_walkers(f1, NW)
    for w in range(NW):
        _, want = oracle.extend(SRC, best_s[w, : info_s["best_r"][w]], 2, mode)
        assert np.array_equal(slots[w, : want.shape[0]], want)
    # result format is not the destination's
    with pytest.raises(tfg.TfgError) as e:
        W.resize(tfg.TFG_RESIZE_EXTEND, 0, f1, 4, axis=1)
    assert e.value.code == tfg.TFG_EINVAL
    # overlapping source and destination in one population
    with pytest.raises(tfg.TfgError) as e:
        W.resize(tfg.TFG_RESIZE_SWAP, 0, 2, 4, index=0)
    assert e.value.code == tfg.TFG_EINVAL
    # range past the population
    with pytest.raises(tfg.TfgError) as e:
        W.resize(tfg.TFG_RESIZE_EXTEND, NW - 2, f1, 4, axis=2)
    assert e.value.code == tfg.TFG_EINVAL
    # a rank-4 aux scheme for (1,2,1) (the naive terms plus a term and its negation):
    # products of rank 4*r exceed r_max = 24 + 3, so every walker is left unchanged
    f2 = W.pop[2]["first"]
    aux = np.concatenate([naive_start(1, 2, 1), [[1, 0, 1, 0, 1], [1, 0, 1, 0, -1]]]).astype(np.int8)
    assert tfg.tfg_verify((1, 2, 1), aux)
    before, _, _ = W.read_walkers(f2, 4)
    assert W.resize(tfg.TFG_RESIZE_PRODUCT, 0, f2, 4, aux=((1, 2, 1), aux)) == 4
    after, _, _ = W.read_walkers(f2, 4)
    assert np.array_equal(before, after)
    W.close()
