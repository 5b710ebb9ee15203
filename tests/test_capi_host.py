"""CPU tests of libtfg's C ABI: every declared symbol is exported, and the host
scheme functions agree with the oracle bit for bit (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2511_20317_gb300 import tfg
from paper_2511_20317_gb300.workloads import golden_dir, naive_start, read_scheme

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_20317_gb300 import _build
    _build.build()
    tfg.lib()


def gold(name):
    return read_scheme(os.path.join(golden_dir(), name))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tfg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tfg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 20
    L = tfg.lib()
    for name in names:
        assert hasattr(L, name), name
    assert sorted(tfg.EXPORTED) == names


def test_verify_fixtures_and_negatives():
    for name in ["paper_2x2x3_r11.txt", "strassen_2x2x2_r7.txt", "paper_sign_example_before.txt"]:
        fmt, s = gold(name)
        assert tfg.tfg_verify(fmt, s)
        s2 = s.copy()
        s2[3, 2] = 1 if s2[3, 2] != 1 else 0
        assert not tfg.tfg_verify(fmt, s2)
    fmt, s = gold("paper_2x2x3_r11.txt")
    assert tfg.tfg_additive_complexity(fmt, s) == 20


def test_error_codes():
    fmt, s = gold("strassen_2x2x2_r7.txt")
    bad = s.copy()
    bad[0, 0] = 2
    with pytest.raises(tfg.TfgError) as e:
        tfg.tfg_prepare(fmt, bad)
    assert e.value.code == tfg.TFG_ESCHEME
    with pytest.raises(tfg.TfgError) as e:
        tfg.tfg_prepare((12, 12, 1), np.zeros((1, 144 + 12 + 12), np.int8))   # a factor of 144 > 128 entries
    assert e.value.code == tfg.TFG_EINVAL
    assert tfg.tfg_verify(fmt, np.abs(s), mode=tfg.TFG_MODE_Z2)    # Strassen reduced mod 2 is a Z_2 scheme
    assert not tfg.tfg_verify(fmt, s, mode=tfg.TFG_MODE_Z2)        # -1 is not a Z_2 coefficient
    with pytest.raises(tfg.TfgError) as e:
        tfg.tfg_project(fmt, s, 0, 5)
    assert e.value.code == tfg.TFG_EINVAL


def test_canonicalize_paper_example():
    fmt, b = gold("paper_sign_example_before.txt")
    _, a = gold("paper_sign_example_after.txt")
    assert np.array_equal(tfg.tfg_canonicalize(fmt, b), a)


@pytest.mark.parametrize("fmt", [(2, 2, 2), (2, 2, 3), (3, 3, 3), (2, 3, 4)])
@pytest.mark.parametrize("mode", [oracle.MODE_ZT, oracle.MODE_Z2])
def test_prepare_matches_oracle(fmt, mode):
    W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(6), seed=4, mode=mode, plateau_len=150).walk(2500)
    rng = np.random.default_rng(0)
    for w in range(6):
        s = W.scheme(w)
        cases = [s, s[::-1].copy()]
        # split a term along w (w = w1 + w2) so that preparation has merges to make
        t = rng.integers(s.shape[0])
        LT = s.shape[1]
        LW = fmt[2] * fmt[0]
        nzw = np.nonzero(s[t, LT - LW:])[0]
        if nzw.size >= 2:
            s2 = np.concatenate([s, s[t:t + 1]])
            first = nzw[0]
            s2[t, LT - LW + first] = 0
            s2[-1, LT - LW:] = 0
            s2[-1, LT - LW + first] = s[t, LT - LW + first]
            assert oracle.brent_valid(fmt, s2, mode)
            cases.append(s2)
        for c in cases:
            a1 = oracle.prepare_start(fmt, c, mode)
            a2 = tfg.tfg_prepare(fmt, c, mode)
            assert np.array_equal(a1, a2)


def test_meta_ops_match_oracle():
    S = gold("strassen_2x2x2_r7.txt")
    E = gold("paper_2x2x3_r11.txt")
    walked = oracle.Walkers((2, 3, 4), naive_start(2, 3, 4), [0], seed=9, plateau_len=300).walk(3000).best_scheme(0)
    W234 = ((2, 3, 4), walked)
    for (fmt, s) in [S, E, W234]:
        for axis in range(3):
            f1, s1 = tfg.tfg_extend(fmt, s, axis)
            f2, s2 = oracle.extend(fmt, s, axis)
            assert f1 == f2 and np.array_equal(s1, s2)
            f1, s1 = tfg.tfg_double(fmt, s, axis)
            f2, s2 = oracle.double(fmt, s, axis)
            assert f1 == f2 and np.array_equal(s1, s2)
            for index in range(fmt[axis]):
                if fmt[axis] < 2:
                    continue
                f1, s1 = tfg.tfg_project(fmt, s, axis, index)
                f2, s2 = oracle.project(fmt, s, axis, index)
                assert f1 == f2 and np.array_equal(s1, s2)
        for perm in range(6):
            f1, s1 = tfg.tfg_swap_sizes(fmt, s, perm)
            f2, s2 = oracle.swap_sizes(fmt, s, perm)
            assert f1 == f2 and np.array_equal(s1, s2)
    f1, s1 = tfg.tfg_product(*S, *S)
    f2, s2 = oracle.product(*S, *S)
    assert f1 == f2 == (4, 4, 4) and np.array_equal(s1, s2) and s1.shape[0] == 49
    f1, s1 = tfg.tfg_product(*E, (1, 2, 1), naive_start(1, 2, 1))
    f2, s2 = oracle.product(*E, (1, 2, 1), naive_start(1, 2, 1))
    assert f1 == f2 and np.array_equal(s1, s2)
    f1, s1 = tfg.tfg_merge(*S, *E, 2)
    f2, s2 = oracle.merge(*S, *E, 2)
    assert f1 == f2 == (2, 2, 5) and np.array_equal(s1, s2)


def test_meta_chain_large_start():
    S = gold("strassen_2x2x2_r7.txt")
    f1, s1 = tfg.tfg_extend(*S, 2)
    f2, s2 = tfg.tfg_double(f1, s1, 2)
    f3, s3 = tfg.tfg_product(*S, f2, s2)
    f4, s4 = tfg.tfg_extend(f3, s3, 1)
    assert f4 == (4, 5, 12) and s4.shape[0] == 202 and tfg.tfg_verify(f4, s4)
    with pytest.raises(tfg.TfgError):
        tfg.tfg_product(f4, s4, *S)   # (8,10,24) exceeds 64 entries per factor


def test_large_format_starts():
    """The meta-operator starts of the large formats: formats, ranks, Eq. (1),
    and the same schemes as the oracle's meta operators produce."""
    from paper_2511_20317_gb300 import starts
    from paper_2511_20317_gb300.workloads import strassen_start
    fmt_s, S = gold("strassen_2x2x2_r7.txt")
    assert np.array_equal(strassen_start(), S)
    for (f, s), want_fmt, want_r in [(starts.start_4_5_12(), (4, 5, 12), 202), (starts.start_5_6_10(), (5, 6, 10), 285),
                                     (starts.start_6_7_9(), (6, 7, 9), 351)]:
        assert f == want_fmt and s.shape[0] == want_r
        assert oracle.brent_valid(f, s)
    # same construction through the oracle's operators
    f1, s1 = oracle.extend(fmt_s, S, 2)
    f2, s2 = oracle.double(f1, s1, 2)
    f3, s3 = oracle.product(fmt_s, S, f2, s2)
    f4, s4 = oracle.extend(f3, s3, 1)
    assert np.array_equal(s4, starts.start_4_5_12()[1])


def test_search_scheme_files_round_trip(tmp_path):
    """The search driver's scheme files read back to the same format and rows."""
    from paper_2511_20317_gb300.search import write_scheme
    for name in ["paper_2x2x3_r11.txt", "strassen_2x2x2_r7.txt"]:
        fmt, s = gold(name)
        path = str(tmp_path / name)
        write_scheme(path, fmt, s, "round trip")
        f2, s2 = read_scheme(path)
        assert f2 == fmt and np.array_equal(s2, s)


def test_lifted_6_7_9_start_from_a_walked_333_scheme():
    """(6,7,9) = extend_n((2,2,3:11) (x) S333): rank 11 r + 54 for any valid (3,3,3)
    scheme S333 of rank r (here one the oracle's walk produced)."""
    from paper_2511_20317_gb300 import starts
    W = oracle.Walkers((3, 3, 3), naive_start(3, 3, 3), np.arange(8), seed=2, plateau_len=400).walk(6000)
    w = int(np.argmin(W.info["best_r"]))
    s333 = W.best_scheme(w)
    fmt, s = starts.start_6_7_9(s333)
    assert fmt == (6, 7, 9) and s.shape[0] == 11 * s333.shape[0] + 54
    assert oracle.brent_valid(fmt, s)


def _poly_dict(t):
    return {tuple(int(v) for v in idx): int(t[idx]) for idx in zip(*np.nonzero(t))}


def test_isotropy_invariants_match_oracle():
    """tfg_isotropy_invariants against the oracle's definitions: term ranks, type
    and symmetric polynomials, rank sums, over Q (Z_T) and GF(2) (Z_2)."""
    from oracle import invariants as inv
    from paper_2511_20317_gb300 import starts
    cases = [gold("strassen_2x2x2_r7.txt"), gold("paper_2x2x3_r11.txt"), ((3, 4, 5), naive_start(3, 4, 5)),
             starts.start_4_5_12()]
    for fmt in [(2, 3, 4), (3, 3, 3), (4, 4, 4)]:
        W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(3), seed=12, plateau_len=400).walk(4000)
        cases += [(fmt, W.best_scheme(w)) for w in range(3)]
    for fmt, s in cases:
        tr, typ, sym, sums = tfg.tfg_isotropy_invariants(fmt, s)
        otr, otyp, osym, osums = inv.isotropy_invariants(fmt, s)
        assert [tuple(t) for t in tr.tolist()] == otr
        assert _poly_dict(typ) == otyp and _poly_dict(sym) == osym and tuple(sums.tolist()) == osums
    for fmt in [(2, 2, 2), (3, 3, 3)]:
        W = oracle.Walkers(fmt, naive_start(*fmt), np.arange(3), seed=5, mode=oracle.MODE_Z2, plateau_len=300).walk(3000)
        for w in range(3):
            s = W.best_scheme(w)
            tr, typ, sym, sums = tfg.tfg_isotropy_invariants(fmt, s, mode=tfg.TFG_MODE_Z2)
            otr, otyp, osym, osums = inv.isotropy_invariants(fmt, s, mode=inv.MODE_Z2)
            assert [tuple(t) for t in tr.tolist()] == otr and _poly_dict(typ) == otyp and tuple(sums.tolist()) == osums
    # full-rank 8 x 8 factors: (8,8,1) naive terms and a dense +-1 test matrix row
    fmt = (8, 8, 1)
    s = naive_start(*fmt)
    rng = np.random.default_rng(3)
    dense = s[:1].copy()
    dense[0, :64] = rng.choice([-1, 1], size=64)
    tr, _, _, _ = tfg.tfg_isotropy_invariants(fmt, dense)
    assert tuple(tr[0]) == inv.term_ranks(fmt, dense)[0]


def test_resize_moves_give_valid_schemes():
    """The Resize moves of the exploratory search (swap sizes, merge with a best
    scheme, project, product, double, extend) on valid schemes give schemes that
    satisfy Eq. (1) (checked by the oracle) and stay within the 128-entry factor limit."""
    from paper_2511_20317_gb300 import search
    from paper_2511_20317_gb300.workloads import strassen_start
    bests = {(2, 2, 2): strassen_start(), (2, 2, 3): gold("paper_2x2x3_r11.txt")[1],
             (2, 3, 3): naive_start(2, 3, 3), (3, 3, 3): naive_start(3, 3, 3)}
    rng = np.random.default_rng(4)
    seen = set()
    for _ in range(300):
        src = list(bests)[int(rng.integers(len(bests)))]
        out = search.resize_move(rng, src, bests[src], bests, p_resize=0.9)
        if out is None:
            continue
        fmt, s, op = out
        seen.add(op.split("+")[-1].rstrip("0123456789"))
        m, n, p = fmt
        assert m * n <= 128 and n * p <= 128 and p * m <= 128
        assert oracle.brent_valid(fmt, s), (src, fmt, op)
    assert {"merge", "product", "double", "extend", "project"} <= seen


@pytest.mark.parametrize("fmt", [(9, 8, 2), (2, 9, 8), (8, 2, 9), (11, 11, 1)])
def test_factors_beyond_64_entries_host(fmt):
    """Factors of 65..128 entries (two 64-bit words): Eq. (1) on the naive scheme
    and on single-coefficient changes, start preparation and the meta operators
    against the oracle, and the isotropy invariants."""
    from oracle import invariants as inv
    s = naive_start(*fmt)
    assert tfg.tfg_verify(fmt, s) and oracle.brent_valid(fmt, s)
    rng = np.random.default_rng(0)
    for _ in range(20):
        bad = s.copy()
        t, e = int(rng.integers(s.shape[0])), int(rng.integers(s.shape[1]))
        bad[t, e] = 0 if bad[t, e] else 1
        assert not tfg.tfg_verify(fmt, bad) and not oracle.brent_valid(fmt, bad)
    W = oracle.Walkers(fmt, s, np.arange(2), seed=3, plateau_len=100).walk(600)
    for w in range(2):
        c = W.scheme(w)
        assert np.array_equal(tfg.tfg_prepare(fmt, c), oracle.prepare_start(fmt, c))
        for axis in range(3):
            if fmt[axis] >= 2:
                f1, s1 = tfg.tfg_project(fmt, c, axis, 1)
                f2, s2 = oracle.project(fmt, c, axis, 1)
                assert f1 == f2 and np.array_equal(s1, s2)
        tr, typ, sym, sums = tfg.tfg_isotropy_invariants(fmt, c)
        otr, otyp, osym, osums = inv.isotropy_invariants(fmt, c)
        assert [tuple(x) for x in tr.tolist()] == otr and _poly_dict(typ) == otyp
