"""Reference oracle for the ternary flip-graph walk.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never imports
it, and it imports nothing from the product package.

Two parts:

* ``oracle.c`` (compiled to ``liboracle.so`` with gcc): Philox4x32-10, the Brent
  check of Eq. (1), sign-symmetry breaking (Section 3.6) and the walker itself
  (Algorithm 1 with the operators of Section 3.3) over int8 arrays.
* this module: a ctypes wrapper and the meta operators of Section 3.3.2
  (project, extend, merge, double, product, swap sizes) written in numpy as
  their plain definitions.

A scheme is an int8 array of shape ``[r, mn + np + pm]``: ``u[i*n+k]`` (a_ik),
``v[k*p+j]`` (b_kj), ``w[j*m+i]`` (c_ij), the C^T convention of Section 3.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_ZT = 0
MODE_Z2 = 1
NOCAND, REJECT, ACCEPT = 0, 1, 2
REFRESH_THRESH_DEFAULT = 42949672  # floor(0.01 * 2**32): the 1% equal-rank refresh of Algorithm 1


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc into liboracle.so next to it."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("plateau_len", ctypes.c_int64),
                ("refresh_thresh", ctypes.c_uint32),
                ("plus_attempts", ctypes.c_int32),
                ("plus_enabled", ctypes.c_int32),
                ("debug_checks", ctypes.c_int32),
                ("policy", ctypes.c_int32),          # 0: plateau plus, 1: Algorithm 1 expansions,
                                                     # 2: additive complexity minimisation
                ("expand_thresh", ctypes.c_uint32)]  # policy 1: p_expand * 2^32


INFO_DTYPE = np.dtype([("r", np.int32), ("best_r", np.int32), ("r_max", np.int32), ("best_nnz", np.int32),
                       ("t", np.int64), ("plateau", np.int64), ("best_t", np.int64),
                       ("digest", np.uint64),
                       ("accepted", np.int64), ("rejected", np.int64), ("nocand", np.int64),
                       ("drops", np.int64), ("merges", np.int64), ("plus", np.int64),
                       ("reductions", np.int64), ("debug_failures", np.int64), ("ops", np.int64)])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_brent_valid.argtypes = [i32, i32, i32, i32, i32, P]
            L.orc_lift_bruteforce.argtypes = [i32, i32, i32, i32, P, i32, P]
            L.orc_lift_backtrack.argtypes = [i32, i32, i32, i32, P, ctypes.c_int64, P]
            L.orc_brent_valid.restype = i32
            L.orc_canonicalize.argtypes = [i32, i32, i32, i32, i32, P]
            L.orc_additive_complexity.argtypes = [i32, i32, i32, i32, P]
            L.orc_additive_complexity.restype = ctypes.c_longlong
            L.orc_prepare_start.argtypes = [i32, i32, i32, i32, i32, P]
            L.orc_prepare_start.restype = i32
            L.orc_enumerate_candidates.argtypes = [i32, i32, i32, i32, i32, P, i32, P]
            L.orc_enumerate_candidates.restype = i32
            L.orc_apply_flip.argtypes = [i32, i32, i32, i32, i32, P, i32, i32, i32, i32, i32, P]
            L.orc_apply_flip.restype = i32
            L.orc_init_walkers.argtypes = [i32, i32, i32, i32, i32, P, i32, i32, P, P, P, P]
            L.orc_walk.argtypes = [i32, i32, i32, i32, ctypes.POINTER(Params), i32, u64,
                                   i32, P, i64, i32, P, P, P]
            L.orc_window_features.argtypes = [i32, i32, i32, i32, i32, P, i32, i32, P, P]
            L.orc_window_features.restype = i32
            L.orc_walk_window.argtypes = [i32, i32, i32, ctypes.POINTER(Params), i32, u64, i32, P, i64, i32,
                                          i32, i32, P, P, P, P, P, P, u32]
            L.orc_digest_init.argtypes = [u32]
            L.orc_digest_init.restype = u64
            L.orc_info_size.restype = i32
            assert L.orc_info_size() == INFO_DTYPE.itemsize
            assert L.orc_params_size() == ctypes.sizeof(Params)
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def term_len(fmt) -> int:
    m, n, p = fmt[:3]
    return m * n + n * p + p * m


# ---------------------------------------------------------------------------------------------
# Primitives
# ---------------------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def brent_valid(fmt, scheme, mode=MODE_ZT) -> bool:
    m, n, p = fmt
    s = np.ascontiguousarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt))
    return bool(lib().orc_brent_valid(m, n, p, mode, s.shape[0], _ptr(s)))


def lift_bruteforce(fmt, z2_scheme, max_bits: int = 24):
    """Every sign assignment (first non-zero of u and v per term +1) of a Z_2
    scheme checked with Eq. (1): (True, signed scheme), (False, None), or None
    when there are more than max_bits free signs."""
    m, n, p = fmt
    s = np.ascontiguousarray(z2_scheme, dtype=np.int8).reshape(-1, term_len(fmt))
    out = np.zeros_like(s)
    rc = lib().orc_lift_bruteforce(m, n, p, s.shape[0], _ptr(s), int(max_bits), _ptr(out))
    if rc < 0:
        return None
    return (True, out) if rc == 1 else (False, None)


def lift_backtrack(fmt, z2_scheme, max_nodes: int = 10**8):
    """Plain backtracking over the free signs, each tensor entry checked with
    Eq. (1) once its signs are set: (True, signed scheme), (False, None), or
    None when the node budget runs out."""
    m, n, p = fmt
    s = np.ascontiguousarray(z2_scheme, dtype=np.int8).reshape(-1, term_len(fmt))
    out = np.zeros_like(s)
    rc = lib().orc_lift_backtrack(m, n, p, s.shape[0], _ptr(s), int(max_nodes), _ptr(out))
    if rc < 0:
        return None
    return (True, out) if rc == 1 else (False, None)


def canonicalize(fmt, scheme, mode=MODE_ZT) -> np.ndarray:
    m, n, p = fmt
    s = np.ascontiguousarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt)).copy()
    lib().orc_canonicalize(m, n, p, mode, s.shape[0], _ptr(s))
    return s


def additive_complexity(fmt, scheme) -> int:
    m, n, p = fmt
    s = np.ascontiguousarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt))
    return int(lib().orc_additive_complexity(m, n, p, s.shape[0], _ptr(s)))


def prepare_start(fmt, scheme, mode=MODE_ZT) -> np.ndarray:
    """Canonicalise, remove terms with a zero factor, apply every reduction."""
    m, n, p = fmt
    s = np.ascontiguousarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt)).copy()
    r = lib().orc_prepare_start(m, n, p, mode, s.shape[0], _ptr(s))
    return s[:r].copy()


def enumerate_candidates(fmt, scheme, i, mode=MODE_ZT) -> np.ndarray:
    """Flip candidates for sampled term i, in walk order: rows (X, j, s, rho)."""
    m, n, p = fmt
    s = np.ascontiguousarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt))
    out = np.zeros((6 * s.shape[0] + 6, 4), dtype=np.int32)
    K = lib().orc_enumerate_candidates(m, n, p, mode, s.shape[0], _ptr(s), int(i), _ptr(out))
    return out[:K].copy()


def apply_flip(fmt, scheme, i, X, j, s, rho, mode=MODE_ZT):
    """Apply one flip candidate to term i, with zero-term removal, sign
    normalisation and the reduction cascade.  Returns (action, new scheme)."""
    m, n, p = fmt
    buf = np.ascontiguousarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt)).copy()
    r_out = ctypes.c_int(0)
    action = lib().orc_apply_flip(m, n, p, mode, buf.shape[0], _ptr(buf), int(i), int(X), int(j),
                                  int(s), int(rho), ctypes.byref(r_out))
    return int(action), buf[: r_out.value].copy()


WINDOW = 256   # candidates per window-mode step (up to 256 candidate pairs per step)


def window_features(fmt, scheme, best_r, i0, W=WINDOW):
    """Window of a state (rank = rows of `scheme`) for start term i0: returns
    (features float32 [K, 32], candidates int32 [K, 5] = (i, X, j, s, rho))."""
    m, n, p = fmt
    s = np.ascontiguousarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt))
    feat = np.zeros((W, 32), np.float32)
    cand = np.zeros((W, 5), np.int32)
    K = lib().orc_window_features(m, n, p, s.shape[0], int(best_r), _ptr(s), int(i0), W, _ptr(feat), _ptr(cand))
    return feat[:K].copy(), cand[:K].copy()


def digest_init(walker_id: int) -> int:
    return int(lib().orc_digest_init(walker_id))


# ---------------------------------------------------------------------------------------------
# Walker population
# ---------------------------------------------------------------------------------------------
class Walkers:
    """A batch of independent walkers of one format, advanced by the C oracle."""

    def __init__(self, fmt, start, walker_ids, seed, *, mode=MODE_ZT, r_slack=3,
                 plateau_len=10_000, refresh_thresh=REFRESH_THRESH_DEFAULT,
                 plus_attempts=16, plus_enabled=True, debug_checks=False, prepared=False,
                 policy=0, expand_thresh=0):
        self.fmt = tuple(int(x) for x in fmt)
        self.mode = int(mode)
        self.LT = term_len(self.fmt)
        st = np.ascontiguousarray(start, dtype=np.int8).reshape(-1, self.LT)
        self.start = st.copy() if prepared else prepare_start(self.fmt, st, mode)
        self.r0 = self.start.shape[0]
        self.r_max = self.r0 + int(r_slack)
        self.seed = int(seed)
        self.walker_ids = np.ascontiguousarray(walker_ids, dtype=np.uint32)
        nw = self.walker_ids.size
        self.params = Params(int(plateau_len), int(refresh_thresh), int(plus_attempts),
                             int(bool(plus_enabled)), int(bool(debug_checks)), int(policy), int(expand_thresh))
        self.slots = np.zeros((nw, self.r_max, self.LT), dtype=np.int8)
        self.best = np.zeros((nw, self.r_max, self.LT), dtype=np.int8)
        self.info = np.zeros(nw, dtype=INFO_DTYPE)
        m, n, p = self.fmt
        lib().orc_init_walkers(m, n, p, self.mode, self.r0, _ptr(self.start), self.r_max, nw,
                               _ptr(self.walker_ids), _ptr(self.slots), _ptr(self.best),
                               _ptr(self.info))

    def walk(self, steps: int, threads: int | None = None):
        if threads is None:
            threads = len(os.sched_getaffinity(0))
        m, n, p = self.fmt
        lib().orc_walk(m, n, p, self.mode, ctypes.byref(self.params), self.r_max, self.seed,
                       self.walker_ids.size, _ptr(self.walker_ids), int(steps), int(threads),
                       _ptr(self.slots), _ptr(self.best), _ptr(self.info))
        return self

    def walk_window(self, steps: int, policy: int = 0, choices=None, window: int = WINDOW,
                    threads: int | None = None, log_neg_thresh: int | None = None):
        """Window-mode steps: policy 0 uniform over the window, policy 1 replays
        choices [n_walkers, steps] (window index per step, -1 = no candidate).
        With log_neg_thresh given, the training-log records of these steps are
        kept in self.log_label [n_walkers, steps] (-1: no record, else the label)
        and self.log_feat [n_walkers, steps, 32] (uint8 features of the chosen
        candidate of every step that had one, recorded or not; self.log_chosen
        marks those steps: feature 31 is one on every candidate)."""
        if threads is None:
            threads = len(os.sched_getaffinity(0))
        m, n, p = self.fmt
        ch = None
        if policy == 1:
            ch = np.ascontiguousarray(choices, dtype=np.int32)
            assert ch.shape == (self.walker_ids.size, steps)
        lab = feat = None
        if log_neg_thresh is not None:
            lab = np.full((self.walker_ids.size, steps), -1, np.int8)
            feat = np.zeros((self.walker_ids.size, steps, 32), np.uint8)
        lib().orc_walk_window(m, n, p, ctypes.byref(self.params), self.r_max, self.seed, self.walker_ids.size,
                              _ptr(self.walker_ids), int(steps), int(threads), int(window), int(policy),
                              _ptr(ch) if ch is not None else None, _ptr(self.slots), _ptr(self.best),
                              _ptr(self.info), _ptr(lab) if lab is not None else None,
                              _ptr(feat) if feat is not None else None,
                              int(log_neg_thresh or 0))
        self.log_label, self.log_feat = lab, feat
        self.log_chosen = None if feat is None else feat[:, :, 31] == 1
        return self

    def scheme(self, w: int) -> np.ndarray:
        return self.slots[w, : self.info["r"][w]].copy()

    def best_scheme(self, w: int) -> np.ndarray:
        return self.best[w, : self.info["best_r"][w]].copy()


def horizon_log(label, feat, chosen, walker_ids, H):
    """Training log with an H-step horizon, from one window walk's per-step
    records (label [walkers, steps]: 1 when the step lowered the rank, 0 for a
    sampled label-0 step, -1 otherwise; feat [walkers, steps, 32]; chosen
    [walkers, steps]: the step had a candidate).  Per walker, in step order: a
    step t that lowered the rank contributes label-1 entries for the chosen
    steps s with t - H < s <= t and s after the walker's previous rank-lowering
    step; a sampled label-0 step contributes itself with label 0.  H = 1 is the
    plain log.  Returns (walker_id, step, label, feat) sorted by walker id,
    step, label."""
    out_w, out_s, out_l, out_f = [], [], [], []
    nw, steps = label.shape
    for w in range(nw):
        last = -1
        for t in range(steps):
            if label[w, t] == 1:
                for s in range(max(t - H + 1, last + 1), t + 1):
                    if chosen[w, s]:
                        out_w.append(walker_ids[w]); out_s.append(s); out_l.append(1.0); out_f.append(feat[w, s])
                last = t
            elif label[w, t] == 0:
                out_w.append(walker_ids[w]); out_s.append(t); out_l.append(0.0); out_f.append(feat[w, t])
    wid = np.array(out_w, np.int64)
    st = np.array(out_s, np.int64)
    lab = np.array(out_l, np.float32)
    f = np.array(out_f, np.uint8).reshape(-1, 32)
    o = np.lexsort((lab, st, wid))
    return wid[o], st[o], lab[o], f[o]


# ---------------------------------------------------------------------------------------------
# Meta operators (Section 3.3.2), plain definitions on int8 arrays.
# Each returns (new_format, new_scheme).  Terms keep their order; new terms follow.
# ---------------------------------------------------------------------------------------------
def split_factors(fmt, scheme):
    m, n, p = fmt
    s = np.asarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt))
    U = s[:, : m * n].reshape(-1, m, n)                      # U[l, i, k]  (a_ik)
    V = s[:, m * n: m * n + n * p].reshape(-1, n, p)         # V[l, k, j]  (b_kj)
    W = s[:, m * n + n * p:].reshape(-1, p, m)               # W[l, j, i]  (c_ij, stored transposed)
    return U, V, W


def join_factors(U, V, W):
    r = U.shape[0]
    return np.concatenate([U.reshape(r, -1), V.reshape(r, -1), W.reshape(r, -1)], axis=1).astype(np.int8)


def _drop_zero_terms(U, V, W):
    keep = [l for l in range(U.shape[0]) if U[l].any() and V[l].any() and W[l].any()]
    return U[keep], V[keep], W[keep]


def project(fmt, scheme, axis, index, mode=MODE_ZT):
    """(m,n,p) -> one dimension minus one: remove row/column `index` along `axis`
    (0: rows of A and C, 1: columns of A and rows of B, 2: columns of B and C),
    then remove terms with a zero factor and restore sign normalisation."""
    U, V, W = split_factors(fmt, scheme)
    m, n, p = fmt
    if axis == 0:
        U = np.delete(U, index, axis=1); W = np.delete(W, index, axis=2); m -= 1
    elif axis == 1:
        U = np.delete(U, index, axis=2); V = np.delete(V, index, axis=1); n -= 1
    else:
        V = np.delete(V, index, axis=2); W = np.delete(W, index, axis=1); p -= 1
    U, V, W = _drop_zero_terms(U, V, W)
    out = join_factors(U, V, W)
    if mode == MODE_ZT:
        out = canonicalize((m, n, p), out, mode)
    return (m, n, p), out


def naive_scheme(fmt) -> np.ndarray:
    """The rank-mnp scheme: one term a_ik * b_kj -> c_ij per (i, k, j)."""
    m, n, p = fmt
    U = np.zeros((m * n * p, m, n), np.int8)
    V = np.zeros((m * n * p, n, p), np.int8)
    W = np.zeros((m * n * p, p, m), np.int8)
    l = 0
    for i in range(m):
        for k in range(n):
            for j in range(p):
                U[l, i, k] = 1; V[l, k, j] = 1; W[l, j, i] = 1
                l += 1
    return join_factors(U, V, W)


def merge(fmt_a, scheme_a, fmt_b, scheme_b, axis, mode=MODE_ZT):
    """Block concatenation along `axis` (0: m, 1: n, 2: p): two schemes that agree
    on the other two sizes compute the two blocks; ranks add.  Section 3.6 keeps
    every scheme sign-normalised after each transformation (Z_T)."""
    Ua, Va, Wa = split_factors(fmt_a, scheme_a)
    Ub, Vb, Wb = split_factors(fmt_b, scheme_b)
    ma, na, pa = fmt_a
    mb, nb, pb = fmt_b
    ra, rb = Ua.shape[0], Ub.shape[0]
    if axis == 0:
        assert na == nb and pa == pb
        m, n, p = ma + mb, na, pa
    elif axis == 1:
        assert ma == mb and pa == pb
        m, n, p = ma, na + nb, pa
    else:
        assert ma == mb and na == nb
        m, n, p = ma, na, pa + pb
    U = np.zeros((ra + rb, m, n), np.int8)
    V = np.zeros((ra + rb, n, p), np.int8)
    W = np.zeros((ra + rb, p, m), np.int8)
    # block a sits at offset 0 on every axis
    U[:ra, :ma, :na] = Ua; V[:ra, :na, :pa] = Va; W[:ra, :pa, :ma] = Wa
    oi = ma if axis == 0 else 0
    ok = na if axis == 1 else 0
    oj = pa if axis == 2 else 0
    U[ra:, oi:oi + mb, ok:ok + nb] = Ub
    V[ra:, ok:ok + nb, oj:oj + pb] = Vb
    W[ra:, oj:oj + pb, oi:oi + mb] = Wb
    out = join_factors(U, V, W)
    if mode == MODE_ZT:
        out = canonicalize((m, n, p), out, mode)
    return (m, n, p), out


def extend(fmt, scheme, axis, mode=MODE_ZT):
    """Add one to a size by merging with the naive scheme of the missing block:
    (m,n,p:r) -> (m,n,p+1 : r+mn) along p, and likewise along m and n."""
    m, n, p = fmt
    block = [(1, n, p), (m, 1, p), (m, n, 1)][axis]
    return merge(fmt, scheme, block, naive_scheme(block), axis, mode)


def double(fmt, scheme, axis, mode=MODE_ZT):
    """Merge a scheme with itself along `axis`."""
    return merge(fmt, scheme, fmt, scheme, axis, mode)


def product(fmt_a, scheme_a, fmt_b, scheme_b, mode=MODE_ZT):
    """Tensor (Kronecker) product: (m1 m2, n1 n2, p1 p2 : r1 r2); term (l1, l2) is
    number l1*r2 + l2; row index i = i1*m2 + i2, and so on for k and j."""
    Ua, Va, Wa = split_factors(fmt_a, scheme_a)
    Ub, Vb, Wb = split_factors(fmt_b, scheme_b)
    m1, n1, p1 = fmt_a
    m2, n2, p2 = fmt_b
    m, n, p = m1 * m2, n1 * n2, p1 * p2
    ra, rb = Ua.shape[0], Ub.shape[0]
    U = np.zeros((ra * rb, m, n), np.int8)
    V = np.zeros((ra * rb, n, p), np.int8)
    W = np.zeros((ra * rb, p, m), np.int8)
    for l1 in range(ra):
        for l2 in range(rb):
            l = l1 * rb + l2
            for i1 in range(m1):
                for i2 in range(m2):
                    for k1 in range(n1):
                        for k2 in range(n2):
                            U[l, i1 * m2 + i2, k1 * n2 + k2] = Ua[l1, i1, k1] * Ub[l2, i2, k2]
            for k1 in range(n1):
                for k2 in range(n2):
                    for j1 in range(p1):
                        for j2 in range(p2):
                            V[l, k1 * n2 + k2, j1 * p2 + j2] = Va[l1, k1, j1] * Vb[l2, k2, j2]
            for j1 in range(p1):
                for j2 in range(p2):
                    for i1 in range(m1):
                        for i2 in range(m2):
                            W[l, j1 * p2 + j2, i1 * m2 + i2] = Wa[l1, j1, i1] * Wb[l2, j2, i2]
    out = join_factors(U, V, W)
    if mode == MODE_ZT:
        out = canonicalize((m, n, p), out, mode)
    return (m, n, p), out


def transpose(fmt, scheme):
    """(AB)^T = B^T A^T: (m,n,p) -> (p,n,m) with u' = v^T, v' = u^T, w' = w^T."""
    U, V, W = split_factors(fmt, scheme)
    m, n, p = fmt
    U2 = np.transpose(V, (0, 2, 1))   # [l, j, k]: a'_jk = b_kj
    V2 = np.transpose(U, (0, 2, 1))   # [l, k, i]: b'_ki = a_ik
    W2 = np.transpose(W, (0, 2, 1))   # [l, i, j]: c'_ji = c_ij, stored as w'[i*p + j]
    return (p, n, m), join_factors(U2, V2, W2)


def cyclic(fmt, scheme):
    """The C^T matmul tensor is invariant under (u, v, w) -> (v, w, u), which maps an
    (m,n,p) scheme to an (n,p,m) scheme without re-indexing."""
    m, n, p = fmt
    U, V, W = split_factors(fmt, scheme)
    r = U.shape[0]
    return (n, p, m), join_factors(V.reshape(r, n, p), W.reshape(r, p, m), U.reshape(r, m, n))


# Target orders of (m, n, p) for swap_sizes(perm): perm 1 is the paper's (m,n,p)->(m,p,n).
SWAP_TARGETS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def swap_sizes(fmt, scheme, perm, mode=MODE_ZT):
    """Reorder the sizes: the result format is tuple(fmt[a] for a in SWAP_TARGETS[perm]).
    Built from `transpose` and `cyclic`; sign normalisation restored afterwards."""
    target = tuple(fmt[a] for a in SWAP_TARGETS[perm])
    f, s = tuple(fmt), np.asarray(scheme, np.int8)
    # search the (at most 6) compositions cyclic^c (transpose^t (S)) for the target order
    for t in range(2):
        ft, st = (transpose(f, s) if t else (f, s))
        for c in range(3):
            order_ok = _order_after(t, c) == SWAP_TARGETS[perm]
            if order_ok:
                out = st
                fo = ft
                for _ in range(c):
                    fo, out = cyclic(fo, out)
                assert fo == target
                if mode == MODE_ZT:
                    out = canonicalize(fo, out, mode)
                return fo, out
    raise ValueError(perm)


def _order_after(t, c):
    order = (0, 1, 2)
    if t:
        order = (order[2], order[1], order[0])
    for _ in range(c):
        order = (order[1], order[2], order[0])
    return order
