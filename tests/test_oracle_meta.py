"""Pins of the meta operators (Section 3.3.2): every output satisfies Eq. (1)
and has the rank the paper states."""
import os

import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300.workloads import golden_dir, naive_start, read_scheme


def gold(name):
    return read_scheme(os.path.join(golden_dir(), name))


STRASSEN = gold("strassen_2x2x2_r7.txt")
EX223 = gold("paper_2x2x3_r11.txt")


def walked(fmt, seed=0, steps=3000):
    W = oracle.Walkers(fmt, naive_start(*fmt), [0], seed=seed, plateau_len=500).walk(steps)
    return W.best_scheme(0)


@pytest.mark.parametrize("mode", [oracle.MODE_ZT, oracle.MODE_Z2])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_extend_rank_formula(axis, mode):
    fmt, s = STRASSEN
    f2, s2 = oracle.extend(fmt, s, axis)
    m, n, p = fmt
    add = [n * p, m * p, m * n][axis]
    assert s2.shape[0] == 7 + add
    assert f2 == tuple(x + (a == axis) for a, x in enumerate(fmt))
    assert oracle.brent_valid(f2, s2, mode)


def test_extend_strassen_gives_rank_11_like_the_paper_example():
    # Section 3.3.2: (m,n,p:r) -> (m,n,p+1:r+mn); (2,2,2:7) -> (2,2,3:11), the
    # rank of the Section 3.1.1 example.
    f2, s2 = oracle.extend(*STRASSEN, 2)
    assert f2 == EX223[0] and s2.shape[0] == EX223[1].shape[0] == 11
    assert oracle.brent_valid(f2, s2)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_merge_and_double(axis):
    fa, sa = STRASSEN
    f2, s2 = oracle.double(fa, sa, axis)
    assert s2.shape[0] == 14 and oracle.brent_valid(f2, s2)
    # merge of two different schemes with matching sizes
    fb = tuple(x + (a == axis) for a, x in enumerate(fa))
    sb = walked(fb)
    f3, s3 = oracle.merge(fa, sa, fb, sb, axis)
    assert s3.shape[0] == 7 + sb.shape[0] and oracle.brent_valid(f3, s3)
    assert f3[axis] == fa[axis] + fb[axis]


def test_product_strassen_squared_is_444_rank_49():
    # Table 5 lists Z_T rank 49 for (4,4,4), which Strassen x Strassen attains.
    f2, s2 = oracle.product(*STRASSEN, *STRASSEN)
    assert f2 == (4, 4, 4) and s2.shape[0] == 49
    assert oracle.brent_valid(f2, s2)
    assert set(np.unique(s2)) <= {-1, 0, 1}


def test_product_mixed_formats():
    fa, sa = EX223
    fb = (1, 2, 1)
    sb = naive_start(*fb)
    f2, s2 = oracle.product(fa, sa, fb, sb)
    assert f2 == (2, 4, 3) and s2.shape[0] == 22 and oracle.brent_valid(f2, s2)


@pytest.mark.parametrize("perm", range(6))
@pytest.mark.parametrize("which", ["ex223", "walked234"])
def test_swap_sizes_all_permutations(perm, which):
    fmt, s = EX223 if which == "ex223" else ((2, 3, 4), walked((2, 3, 4), seed=3))
    f2, s2 = oracle.swap_sizes(fmt, s, perm)
    assert f2 == tuple(fmt[a] for a in oracle.SWAP_TARGETS[perm])
    assert s2.shape[0] == s.shape[0]
    assert oracle.brent_valid(f2, s2)
    assert np.array_equal(oracle.canonicalize(f2, s2), s2)


def test_paper_swap_is_m_p_n():
    # Section 3.3.2: swap sizes maps (m, n, p: r) to (m, p, n: r).
    f2, s2 = oracle.swap_sizes(*EX223, 1)
    assert f2 == (2, 3, 2) and oracle.brent_valid(f2, s2)


def test_transpose_and_cycle_orders():
    fmt, s = EX223
    f1, s1 = oracle.transpose(*oracle.transpose(fmt, s))
    assert f1 == fmt and np.array_equal(s1, s)
    f3, s3 = oracle.cyclic(*oracle.cyclic(*oracle.cyclic(fmt, s)))
    assert f3 == fmt and np.array_equal(s3, s)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_project(axis):
    fmt = (3, 3, 3)
    s = walked(fmt, seed=5, steps=4000)
    for index in range(3):
        f2, s2 = oracle.project(fmt, s, axis, index)
        assert f2[axis] == 2
        assert s2.shape[0] <= s.shape[0]
        assert oracle.brent_valid(f2, s2)
    # projecting the naive scheme removes exactly the terms that touch the index
    f2, s2 = oracle.project(fmt, naive_start(*fmt), axis, 1)
    assert s2.shape[0] == 18 and oracle.brent_valid(f2, s2)


def test_meta_chain_for_large_formats():
    """Starts for the large formats are built by chains of meta operators; each
    intermediate is a valid scheme of the predicted rank."""
    f1, s1 = oracle.extend(*STRASSEN, 2)                 # (2,2,3:11)
    f2, s2 = oracle.double(f1, s1, 2)                    # (2,2,6:22)
    f3, s3 = oracle.product(*STRASSEN, f2, s2)           # (4,4,12:154)
    assert f3 == (4, 4, 12) and s3.shape[0] == 154 and oracle.brent_valid(f3, s3)
    f4, s4 = oracle.extend(f3, s3, 1)                    # (4,5,12:154+48)
    assert f4 == (4, 5, 12) and s4.shape[0] == 202 and oracle.brent_valid(f4, s4)
