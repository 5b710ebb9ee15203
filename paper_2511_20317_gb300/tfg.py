"""Python binding of libtfg (include/tfg.h): argument marshalling only.

Every function named ``tfg_*`` here calls the C function of the same name.
PyTorch provides the device workspace and the CUDA stream; every step of the
walk runs in the library's CUDA kernels.  There is no CPU fallback: if
libtfg.so is missing or CUDA is unavailable, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtfg.so")

TFG_OK, TFG_EINVAL, TFG_ESCHEME, TFG_ENOSPC, TFG_ENOMEM, TFG_ECUDA, TFG_ETIMEOUT, TFG_EINTERNAL = 0, -1, -2, -3, -4, -5, -6, -7
TFG_MODE_ZT, TFG_MODE_Z2 = 0, 1
ERROR_NAMES = {0: "TFG_OK", -1: "TFG_EINVAL", -2: "TFG_ESCHEME", -3: "TFG_ENOSPC", -4: "TFG_ENOMEM",
               -5: "TFG_ECUDA", -6: "TFG_ETIMEOUT", -7: "TFG_EINTERNAL"}


class TfgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class tfg_format(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("p", ctypes.c_int32), ("mode", ctypes.c_int32)]


class tfg_params(ctypes.Structure):
    _fields_ = [("plateau_len", ctypes.c_int64), ("refresh_thresh", ctypes.c_uint32),
                ("plus_attempts", ctypes.c_int32), ("plus_enabled", ctypes.c_int32),
                ("r_slack", ctypes.c_int32), ("mapping", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("walker_id_base", ctypes.c_uint32),
                ("use_graph", ctypes.c_int32), ("walk_policy", ctypes.c_int32),
                ("expand_thresh", ctypes.c_uint32), ("reserved", ctypes.c_int32 * 2)]


class tfg_resize_args(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("axis", ctypes.c_int32), ("index", ctypes.c_int32),
                ("use_best", ctypes.c_int32), ("src_first", ctypes.c_int64), ("dst_first", ctypes.c_int64),
                ("count", ctypes.c_int64), ("aux_fmt", tfg_format), ("aux_rank", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("aux_scheme", ctypes.c_void_p)]


TFG_RESIZE_PROJECT, TFG_RESIZE_EXTEND, TFG_RESIZE_DOUBLE, TFG_RESIZE_MERGE, TFG_RESIZE_PRODUCT, TFG_RESIZE_SWAP = range(6)


class tfg_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("walkers", "steps", "accepted", "rejected", "nocand", "drops",
                                              "merges", "plus", "reductions")] + \
               [("min_best_r", ctypes.c_int32), ("max_best_r", ctypes.c_int32)]


class tfg_log_spec(ctypes.Structure):
    _fields_ = [("d_entries", ctypes.c_void_p), ("capacity", ctypes.c_int64), ("d_count", ctypes.c_void_p),
                ("neg_thresh", ctypes.c_uint32), ("horizon", ctypes.c_int32), ("d_ring", ctypes.c_void_p),
                ("d_ring_step", ctypes.c_void_p)]


LOG_ENTRY_DTYPE = np.dtype([("feat", np.uint16, 32), ("label", np.float32), ("walker_id", np.uint32),
                            ("step", np.uint32), ("pad", np.uint32)])
WINDOW = 256
MLP_NUM_PARAMS = 32 * 128 + 128 * 128 + 3 * 128 + 1   # W1, W2, b1, b2, w3, b3 of the proposal network

WALKER_INFO_DTYPE = np.dtype([("r", np.int32), ("best_r", np.int32), ("r_max", np.int32), ("format", np.int32),
                              ("t", np.int64), ("plateau", np.int64), ("best_t", np.int64),
                              ("digest", np.uint64),
                              ("accepted", np.int64), ("rejected", np.int64), ("nocand", np.int64),
                              ("drops", np.int64), ("merges", np.int64), ("plus", np.int64),
                              ("reductions", np.int64), ("walker_id", np.uint32), ("best_nnz", np.uint32)])

# every symbol include/tfg.h declares
EXPORTED = ["tfg_default_params", "tfg_last_error", "tfg_verify", "tfg_additive_complexity", "tfg_isotropy_invariants",
            "tfg_lift_signs", "tfg_canonicalize",
            "tfg_prepare", "tfg_project", "tfg_extend", "tfg_merge", "tfg_double", "tfg_product",
            "tfg_swap_sizes", "tfg_workspace_size", "tfg_init", "tfg_walk", "tfg_sync", "tfg_collect_best",
            "tfg_verify_all_async", "tfg_stats_get", "tfg_read_walkers", "tfg_reseed", "tfg_resize_scratch_bytes",
            "tfg_resize", "tfg_population",
            "tfg_checkpoint",
            "tfg_restore", "tfg_mapping", "tfg_autotune", "tfg_destroy", "tfg_philox_device", "tfg_mlp_param_bytes",
            "tfg_mlp_score", "tfg_mlp_grad", "tfg_mlp_train_state_bytes", "tfg_mlp_train_init",
            "tfg_mlp_train_step", "tfg_window_scratch_bytes", "tfg_walk_window", "tfg_walk_window_noalloc",
            "tfg_test_set_wait_limit", "tfg_window_dump", "tfg_launch_shape"]

_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load libtfg.so (built by __graft_entry__.build() or paper_2511_20317_gb300._build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libtfg.so not built ({LIB_PATH}); run paper_2511_20317_gb300._build.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64, u32, u64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                         ctypes.c_uint64, ctypes.c_size_t)
            F = ctypes.POINTER(tfg_format)
            sig = {
                "tfg_default_params": (None, [ctypes.POINTER(tfg_params)]),
                "tfg_last_error": (ctypes.c_char_p, []),
                "tfg_verify": (i32, [F, i32, P]),
                "tfg_additive_complexity": (i32, [F, i32, P, ctypes.POINTER(ctypes.c_int64)]),
                "tfg_isotropy_invariants": (i32, [F, i32, P, P, P, P, P]),
                "tfg_lift_signs": (i32, [F, i32, P, i64, P, ctypes.POINTER(ctypes.c_int64)]),
                "tfg_canonicalize": (i32, [F, i32, P]),
                "tfg_prepare": (i32, [F, i32, P, P, i32, ctypes.POINTER(ctypes.c_int32)]),
                "tfg_project": (i32, [F, i32, P, i32, i32, F, P, i32, ctypes.POINTER(ctypes.c_int32)]),
                "tfg_extend": (i32, [F, i32, P, i32, F, P, i32, ctypes.POINTER(ctypes.c_int32)]),
                "tfg_merge": (i32, [F, i32, P, F, i32, P, i32, F, P, i32, ctypes.POINTER(ctypes.c_int32)]),
                "tfg_double": (i32, [F, i32, P, i32, F, P, i32, ctypes.POINTER(ctypes.c_int32)]),
                "tfg_product": (i32, [F, i32, P, F, i32, P, F, P, i32, ctypes.POINTER(ctypes.c_int32)]),
                "tfg_swap_sizes": (i32, [F, i32, P, i32, F, P, i32, ctypes.POINTER(ctypes.c_int32)]),
                "tfg_workspace_size": (i32, [i32, F, P, P, ctypes.POINTER(tfg_params), ctypes.POINTER(sz)]),
                "tfg_init": (i32, [i32, F, P, P, P, u64, ctypes.POINTER(tfg_params), P, sz, P,
                                   ctypes.POINTER(P)]),
                "tfg_walk": (i32, [P, i64]),
                "tfg_sync": (i32, [P]),
                "tfg_collect_best": (i32, [P, i32, P, i32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int64)]),
                "tfg_verify_all_async": (i32, [P, P]),
                "tfg_stats_get": (i32, [P, i32, ctypes.POINTER(tfg_stats), P, i32]),
                "tfg_read_walkers": (i32, [P, i64, i64, P, P, P, i32]),
                "tfg_reseed": (i32, [P, i64, i64, i32, P]),
                "tfg_resize_scratch_bytes": (sz, [i32, F, F]),
                "tfg_resize": (i32, [P, ctypes.POINTER(tfg_resize_args), P, sz, ctypes.POINTER(ctypes.c_int64)]),
                "tfg_population": (i32, [P, i32, F, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
                "tfg_checkpoint": (i32, [P, P, sz, ctypes.POINTER(sz)]),
                "tfg_restore": (i32, [P, P, sz]),
                "tfg_mapping": (i32, [P, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
                "tfg_destroy": (None, [P]),
                "tfg_autotune": (i32, [P, i64, i64, P]),
                "tfg_philox_device": (i32, [P, i32, u32, u32, P, P]),
                "tfg_mlp_param_bytes": (sz, []),
                "tfg_mlp_score": (i32, [P, P, i64, P, P, P]),
                "tfg_mlp_grad": (i32, [P, P, P, P, i64, P, P, P]),
                "tfg_window_scratch_bytes": (i32, [P, ctypes.POINTER(sz)]),
                "tfg_walk_window_noalloc": (i32, [P, i64, i32, P, ctypes.c_uint32, P,
                                                  ctypes.POINTER(tfg_log_spec)]),
                "tfg_walk_window": (i32, [P, i64, i32, P, ctypes.c_uint32, P, sz, P, ctypes.POINTER(tfg_log_spec)]),
                "tfg_mlp_train_state_bytes": (sz, []),
                "tfg_mlp_train_init": (i32, [P, P, P]),
                "tfg_mlp_train_step": (i32, [P, P, P, P, P, i64, ctypes.c_float, i32, P, P]),
                "tfg_test_set_wait_limit": (None, [i64]),
                "tfg_window_dump": (i32, [P, P, P, P]),
                "tfg_launch_shape": (i32, [P, i32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int64)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != TFG_OK:
        raise TfgError(rc, lib().tfg_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fmt(fmt, mode=TFG_MODE_ZT) -> tfg_format:
    if isinstance(fmt, tfg_format):
        return fmt
    m, n, p = fmt[:3]
    return tfg_format(int(m), int(n), int(p), int(fmt[3] if len(fmt) > 3 else mode))


def term_len(fmt) -> int:
    m, n, p = fmt[:3]
    return m * n + n * p + p * m


def _rows(fmt, scheme) -> np.ndarray:
    return np.ascontiguousarray(scheme, dtype=np.int8).reshape(-1, term_len(fmt))


# ---------------------------------------------------------------------------------------------
# host functions
# ---------------------------------------------------------------------------------------------
def tfg_default_params(**overrides) -> tfg_params:
    p = tfg_params()
    lib().tfg_default_params(ctypes.byref(p))
    names = {f[0] for f in tfg_params._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"tfg_params has no field {k!r}")
        setattr(p, k, v)
    return p


def tfg_verify(fmt, scheme, mode=TFG_MODE_ZT) -> bool:
    s = _rows(fmt, scheme)
    rc = lib().tfg_verify(ctypes.byref(_fmt(fmt, mode)), s.shape[0], _ptr(s))
    if rc in (TFG_OK, TFG_ESCHEME):
        return rc == TFG_OK
    _check(rc)


def tfg_additive_complexity(fmt, scheme) -> int:
    s = _rows(fmt, scheme)
    out = ctypes.c_int64()
    _check(lib().tfg_additive_complexity(ctypes.byref(_fmt(fmt)), s.shape[0], _ptr(s), ctypes.byref(out)))
    return out.value


def tfg_isotropy_invariants(fmt, scheme, mode=TFG_MODE_ZT):
    """(term ranks int32 [r, 3], type polynomial int64 [12, 12, 12], symmetric
    polynomial int64 [12, 12, 12], rank sums int64 [3])."""
    s = _rows(fmt, scheme)
    tr = np.zeros((s.shape[0], 3), dtype=np.int32)
    typ = np.zeros((12, 12, 12), dtype=np.int64)
    sym = np.zeros((12, 12, 12), dtype=np.int64)
    sums = np.zeros(3, dtype=np.int64)
    _check(lib().tfg_isotropy_invariants(ctypes.byref(_fmt(fmt, mode)), s.shape[0], _ptr(s), _ptr(tr), _ptr(typ),
                                         _ptr(sym), _ptr(sums)))
    return tr, typ, sym, sums


def tfg_lift_signs(fmt, scheme, max_nodes: int = 10**7):
    """Signed (Z_T) scheme with the non-zero pattern of the Z_2 scheme, and the
    search nodes used.  Raises TfgError (TFG_ESCHEME: no sign assignment exists;
    TFG_ETIMEOUT: budget exhausted)."""
    s = _rows(fmt, scheme)
    out = np.zeros_like(s)
    nodes = ctypes.c_int64()
    _check(lib().tfg_lift_signs(ctypes.byref(_fmt(fmt, TFG_MODE_Z2)), s.shape[0], _ptr(s), int(max_nodes), _ptr(out),
                                ctypes.byref(nodes)))
    return out, nodes.value


def polynomial_terms(coeffs) -> dict:
    """{(a, b, c): coefficient} of the non-zero entries of a [12, 12, 12] table."""
    return {tuple(int(v) for v in idx): int(coeffs[idx]) for idx in zip(*np.nonzero(coeffs))}


def tfg_canonicalize(fmt, scheme, mode=TFG_MODE_ZT) -> np.ndarray:
    s = _rows(fmt, scheme).copy()
    _check(lib().tfg_canonicalize(ctypes.byref(_fmt(fmt, mode)), s.shape[0], _ptr(s)))
    return s


def tfg_prepare(fmt, scheme, mode=TFG_MODE_ZT) -> np.ndarray:
    s = _rows(fmt, scheme)
    out = np.zeros_like(s)
    r = ctypes.c_int32()
    _check(lib().tfg_prepare(ctypes.byref(_fmt(fmt, mode)), s.shape[0], _ptr(s), _ptr(out), s.shape[0],
                             ctypes.byref(r)))
    return out[: r.value].copy()


def _meta_call(name, args, cap_terms, out_lt_max=3 * 128):
    # the library writes cap_terms rows of the result format's length (at most
    # three factors of 128 entries)
    out_fmt = tfg_format()
    out = np.zeros((max(cap_terms, 1), out_lt_max), dtype=np.int8)
    r = ctypes.c_int32()
    _check(getattr(lib(), name)(*args, ctypes.byref(out_fmt), _ptr(out), max(cap_terms, 1), ctypes.byref(r)))
    f = (out_fmt.m, out_fmt.n, out_fmt.p)
    LT = term_len(f)
    # the library wrote rows of LT entries contiguously
    flat = out.reshape(-1)[: r.value * LT].reshape(r.value, LT).copy()
    return f, flat


def tfg_project(fmt, scheme, axis, index, mode=TFG_MODE_ZT):
    s = _rows(fmt, scheme)
    return _meta_call("tfg_project", [ctypes.byref(_fmt(fmt, mode)), s.shape[0], _ptr(s), axis, index], s.shape[0])


def tfg_extend(fmt, scheme, axis, mode=TFG_MODE_ZT):
    s = _rows(fmt, scheme)
    m, n, p = fmt[:3]
    cap = s.shape[0] + [n * p, m * p, m * n][axis]
    return _meta_call("tfg_extend", [ctypes.byref(_fmt(fmt, mode)), s.shape[0], _ptr(s), axis], cap)


def tfg_merge(fmt_a, scheme_a, fmt_b, scheme_b, axis, mode=TFG_MODE_ZT):
    a, b = _rows(fmt_a, scheme_a), _rows(fmt_b, scheme_b)
    return _meta_call("tfg_merge", [ctypes.byref(_fmt(fmt_a, mode)), a.shape[0], _ptr(a),
                                    ctypes.byref(_fmt(fmt_b, mode)), b.shape[0], _ptr(b), axis],
                      a.shape[0] + b.shape[0])


def tfg_double(fmt, scheme, axis, mode=TFG_MODE_ZT):
    s = _rows(fmt, scheme)
    return _meta_call("tfg_double", [ctypes.byref(_fmt(fmt, mode)), s.shape[0], _ptr(s), axis], 2 * s.shape[0])


def tfg_product(fmt_a, scheme_a, fmt_b, scheme_b, mode=TFG_MODE_ZT):
    a, b = _rows(fmt_a, scheme_a), _rows(fmt_b, scheme_b)
    return _meta_call("tfg_product", [ctypes.byref(_fmt(fmt_a, mode)), a.shape[0], _ptr(a),
                                      ctypes.byref(_fmt(fmt_b, mode)), b.shape[0], _ptr(b)],
                      a.shape[0] * b.shape[0])


def tfg_swap_sizes(fmt, scheme, perm, mode=TFG_MODE_ZT):
    s = _rows(fmt, scheme)
    return _meta_call("tfg_swap_sizes", [ctypes.byref(_fmt(fmt, mode)), s.shape[0], _ptr(s), perm], s.shape[0])


def tfg_philox_device(ctr: np.ndarray, key_lo: int, key_hi: int) -> np.ndarray:
    import torch
    c = torch.from_numpy(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32)).cuda()
    out = torch.empty_like(c)
    _check(lib().tfg_philox_device(ctypes.c_void_p(c.data_ptr()), c.numel() // 4, key_lo, key_hi,
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return out.cpu().numpy().view(np.uint32)


def tfg_mlp_param_bytes() -> int:
    return int(lib().tfg_mlp_param_bytes())


def tfg_mlp_score(params, x, out=None, err=None, stream=None):
    """Score candidate rows x (torch bf16 [n, 32] on the device) with the MLP whose
    parameter blob `params` is a torch uint8 device tensor; returns f32 scores."""
    import torch
    n = x.shape[0]
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=x.device)
    own_err = err is None
    if own_err:
        err = torch.zeros(1, dtype=torch.int32, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().tfg_mlp_score(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(x.data_ptr()), n,
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(err.data_ptr()),
                               ctypes.c_void_p(st.cuda_stream)))
    if own_err:
        if int(err.item()) != 0:
            raise TfgError(TFG_ETIMEOUT, "tensor-core completion wait gave up")
    return out


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def tfg_mlp_grad(params, x, label, weight, stream=None):
    """Gradient (float32 [P]) and loss of the weighted logistic loss on (x, label, weight)."""
    import torch
    P = MLP_NUM_PARAMS
    grad = torch.empty(P + 1, dtype=torch.float32, device=x.device)
    err = torch.zeros(1, dtype=torch.int32, device=x.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().tfg_mlp_grad(_vp(params), _vp(x), _vp(label), _vp(weight), x.shape[0], _vp(grad), _vp(err),
                              ctypes.c_void_p(st.cuda_stream)))
    if int(err.item()) != 0:
        raise TfgError(TFG_ETIMEOUT, "tensor-core completion wait gave up")
    return grad[:P], float(grad[P].item())


def tfg_test_set_wait_limit(polls: int):
    """Test hook: poll limit of the scoring network's first completion wait per CTA
    (negative restores the default)."""
    lib().tfg_test_set_wait_limit(int(polls))


def tfg_mlp_train_state_bytes() -> int:
    return int(lib().tfg_mlp_train_state_bytes())


class TransitionLog:
    """Device buffers for window-mode logging (entries, count), read back as numpy.
    With horizon > 1 it also holds the walkers' rings of recent chosen
    candidates, which carry over between calls: use one log per context."""

    def __init__(self, capacity: int, neg_thresh: int = 0, horizon: int = 1):
        import torch
        self.capacity = int(capacity)
        self.neg_thresh = int(neg_thresh)
        self.horizon = int(horizon)
        self.entries = torch.zeros(self.capacity * LOG_ENTRY_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        self.count = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.ring = self.ring_step = None   # horizon > 1: per-walker rings, made at the first walk

    def spec(self, walkers: int) -> "tfg_log_spec":
        import torch
        ring = step = None
        if self.horizon > 1:
            if self.ring is None or self.ring_step.numel() != walkers * self.horizon:
                self.ring = torch.zeros(walkers * self.horizon * 32, dtype=torch.int16, device="cuda")
                self.ring_step = torch.full((walkers * self.horizon,), -1, dtype=torch.int32, device="cuda")
            ring, step = self.ring.data_ptr(), self.ring_step.data_ptr()
        return tfg_log_spec(self.entries.data_ptr(), self.capacity, self.count.data_ptr(), self.neg_thresh,
                            self.horizon, ring, step)

    def read(self) -> np.ndarray:
        n = min(int(self.count.item()), self.capacity)
        return self.entries[: n * LOG_ENTRY_DTYPE.itemsize].cpu().numpy().view(LOG_ENTRY_DTYPE).copy()


class MlpTrainer:
    """Adam training of the parameter blob `params` (torch uint8 device tensor, updated in place)."""

    def __init__(self, params, stream=None):
        import torch
        self.params = params
        self.state = torch.zeros(tfg_mlp_train_state_bytes() // 4, dtype=torch.float32, device=params.device)
        self.err = torch.zeros(1, dtype=torch.int32, device=params.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.step_no = 0
        _check(lib().tfg_mlp_train_init(_vp(self.state), _vp(params), ctypes.c_void_p(self.stream.cuda_stream)))

    def tfg_mlp_train_step(self, x, label, weight, lr):
        self.step_no += 1
        _check(lib().tfg_mlp_train_step(_vp(self.state), _vp(self.params), _vp(x), _vp(label), _vp(weight),
                                        x.shape[0], ctypes.c_float(lr), self.step_no, _vp(self.err),
                                        ctypes.c_void_p(self.stream.cuda_stream)))

    step = tfg_mlp_train_step

    def loss(self) -> float:
        P = MLP_NUM_PARAMS
        return float(self.state[3 * P + P].item())   # the loss follows the gradient


# ---------------------------------------------------------------------------------------------
# walker contexts
# ---------------------------------------------------------------------------------------------
class Walkers:
    """A context of walker populations on the current CUDA device.

    populations: list of (fmt (m,n,p), mode, start scheme int8 [r, LT], n_walkers).
    The device workspace is a torch uint8 tensor owned by this object; all work
    is ordered on `stream` (default: torch's current stream)."""

    def __init__(self, populations, seed: int, params: tfg_params | None = None, stream=None):
        import torch
        self.torch = torch
        L = lib()
        self.params = params if params is not None else tfg_default_params()
        nf = len(populations)
        self.fmts = (tfg_format * nf)()
        prepared, ranks, walkers = [], (ctypes.c_int32 * nf)(), (ctypes.c_int64 * nf)()
        for a, (fmt, mode, start, nw) in enumerate(populations):
            self.fmts[a] = _fmt(fmt, mode)
            st = tfg_prepare(fmt, start, mode)  # validates and reports the prepared rank
            prepared.append(_rows(fmt, start))
            ranks[a] = st.shape[0]
            walkers[a] = int(nw)
        self._starts = prepared
        in_ranks = (ctypes.c_int32 * nf)(*[s.shape[0] for s in prepared])
        bytes_ = ctypes.c_size_t()
        _check(L.tfg_workspace_size(nf, self.fmts, ctypes.cast(ranks, ctypes.c_void_p),
                                    ctypes.cast(walkers, ctypes.c_void_p), ctypes.byref(self.params),
                                    ctypes.byref(bytes_)))
        self.workspace_bytes = bytes_.value
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device="cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ptrs = (ctypes.c_void_p * nf)(*[s.ctypes.data for s in prepared])
        ctx = ctypes.c_void_p()
        _check(L.tfg_init(nf, self.fmts, ctypes.cast(in_ranks, ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p),
                          ctypes.cast(walkers, ctypes.c_void_p), ctypes.c_uint64(seed), ctypes.byref(self.params),
                          ctypes.c_void_p(self.workspace.data_ptr()), self.workspace_bytes,
                          ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx)))
        self.ctx = ctx
        self.n_formats = nf
        self.pop = [self.population(a) for a in range(nf)]
        self.total = sum(p["walkers"] for p in self.pop)

    # -- plain calls ----------------------------------------------------------
    def tfg_walk(self, steps: int):
        _check(lib().tfg_walk(self.ctx, int(steps)))
        return self

    walk = tfg_walk

    def tfg_sync(self):
        _check(lib().tfg_sync(self.ctx))
        return self

    sync = tfg_sync

    def population(self, f: int) -> dict:
        fmt, r0, rmax, nw, first = tfg_format(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().tfg_population(self.ctx, f, ctypes.byref(fmt), ctypes.byref(r0), ctypes.byref(rmax),
                                    ctypes.byref(nw), ctypes.byref(first)))
        G, S, SL, SQ = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().tfg_mapping(self.ctx, f, ctypes.byref(G), ctypes.byref(S), ctypes.byref(SL), ctypes.byref(SQ)))
        BT, GR = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().tfg_launch_shape(self.ctx, f, None, ctypes.byref(BT), ctypes.byref(GR)))
        return {"fmt": (fmt.m, fmt.n, fmt.p), "mode": fmt.mode, "r0": r0.value, "r_max": rmax.value,
                "walkers": nw.value, "first": first.value, "lanes": G.value, "slots_per_lane": S.value,
                "slice_len": SL.value, "square": SQ.value, "block_threads": BT.value, "grid": GR.value}

    def tfg_autotune(self, trial_steps: int = 400, trial_walkers: int = 32768):
        lanes = (ctypes.c_int32 * self.n_formats)()
        _check(lib().tfg_autotune(self.ctx, int(trial_steps), int(trial_walkers), ctypes.cast(lanes, ctypes.c_void_p)))
        self.pop = [self.population(a) for a in range(self.n_formats)]
        return list(lanes)

    autotune = tfg_autotune

    def tfg_collect_best(self, f: int):
        p = self.pop[f]
        out = np.zeros((p["r_max"], term_len(p["fmt"])), dtype=np.int8)
        r, w = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().tfg_collect_best(self.ctx, f, _ptr(out), p["r_max"], ctypes.byref(r), ctypes.byref(w)))
        return out[: r.value].copy(), r.value, w.value

    collect_best = tfg_collect_best

    def tfg_verify_all(self) -> int:
        fails = self.torch.zeros(1, dtype=self.torch.int64, device="cuda")
        _check(lib().tfg_verify_all_async(self.ctx, ctypes.c_void_p(fails.data_ptr())))
        self.sync()
        return int(fails.item())

    verify_all = tfg_verify_all

    def tfg_stats_get(self, f: int = -1, hist_len: int = 1024):
        st = tfg_stats()
        hist = np.zeros(hist_len, dtype=np.int64)
        _check(lib().tfg_stats_get(self.ctx, f, ctypes.byref(st), _ptr(hist), hist_len))
        d = {k: getattr(st, k) for k, _ in tfg_stats._fields_}
        return d, hist

    stats = tfg_stats_get

    def tfg_read_walkers(self, first: int, count: int, slots: bool = True, best: bool = True):
        """Returns (info structured array, slots int8 [count, r_max, LT] | None, best | None)."""
        f = next(a for a, p in enumerate(self.pop) if p["first"] <= first < p["first"] + p["walkers"])
        p = self.pop[f]
        LT = term_len(p["fmt"])
        info = np.zeros(count, dtype=WALKER_INFO_DTYPE)
        s = np.zeros((count, p["r_max"], LT), dtype=np.int8) if slots else None
        b = np.zeros((count, p["r_max"], LT), dtype=np.int8) if best else None
        _check(lib().tfg_read_walkers(self.ctx, first, count, _ptr(info),
                                      _ptr(s) if slots else None, _ptr(b) if best else None, p["r_max"]))
        return info, s, b

    read_walkers = tfg_read_walkers

    def tfg_reseed(self, first: int, count: int, scheme):
        """Replace walkers [first, first + count) of one population by `scheme`."""
        f = next(a for a, p in enumerate(self.pop) if p["first"] <= first < p["first"] + p["walkers"])
        s = _rows(self.pop[f]["fmt"], scheme)
        _check(lib().tfg_reseed(self.ctx, int(first), int(count), s.shape[0], _ptr(s)))
        return self

    reseed = tfg_reseed

    def tfg_resize(self, op: int, src_first: int, dst_first: int, count: int, axis: int = 0, index: int = 0,
                   aux=None, use_best: bool = False) -> int:
        """Device resize: walkers [src_first, +count) transformed by meta operator `op`
        (TFG_RESIZE_*) into walkers [dst_first, +count) of the result format's
        population; aux = (fmt, scheme) for merge / product.  Returns the number of
        walkers left unchanged because their result exceeds the destination's r_max
        (the library's TFG_ENOSPC); every other error raises TfgError."""
        a = tfg_resize_args()
        a.op, a.axis, a.index, a.use_best = int(op), int(axis), int(index), int(bool(use_best))
        a.src_first, a.dst_first, a.count = int(src_first), int(dst_first), int(count)
        rows = None
        src_mode = next(p["mode"] for p in self.pop if p["first"] <= src_first < p["first"] + p["walkers"])
        if aux is not None:
            afmt, ascheme = aux
            rows = _rows(tuple(afmt), ascheme)
            a.aux_fmt = tfg_format(*afmt, src_mode)
            a.aux_rank = rows.shape[0]
            a.aux_scheme = rows.ctypes.data
        dst = next(p for p in self.pop if p["first"] <= dst_first < p["first"] + p["walkers"])
        out = tfg_format(*dst["fmt"], dst["mode"])
        need = lib().tfg_resize_scratch_bytes(a.aux_rank, ctypes.byref(a.aux_fmt) if rows is not None else None,
                                              ctypes.byref(out))
        torch = self.torch
        if getattr(self, "_rscratch", None) is None or self._rscratch.numel() < need:
            self._rscratch = torch.empty(max(int(need), 1), dtype=torch.uint8, device="cuda")
        skipped = ctypes.c_int64(0)
        rc = lib().tfg_resize(self.ctx, ctypes.byref(a), ctypes.c_void_p(self._rscratch.data_ptr()),
                              self._rscratch.numel(), ctypes.byref(skipped))
        if rc == TFG_ENOSPC and skipped.value > 0:
            return int(skipped.value)
        _check(rc)
        return 0

    resize = tfg_resize

    def tfg_walk_window(self, steps: int, policy: int = 0, mlp_params=None, eps_thresh: int = 0,
                        record_choices: bool = False, log=None):
        """Window-mode steps (policy 0 uniform over the window, 1 learned).  Returns
        the chosen window indices [steps, walkers] (device tensor) when asked."""
        torch = self.torch
        if getattr(self, "_wscratch", None) is None:
            b = ctypes.c_size_t()
            _check(lib().tfg_window_scratch_bytes(self.ctx, ctypes.byref(b)))
            self._wscratch = torch.empty(b.value, dtype=torch.uint8, device="cuda")
        choices = None
        if record_choices:
            choices = torch.full((steps, self.total), -2, dtype=torch.int32, device="cuda")
        spec = None
        if log is not None:
            spec = log.spec(self.total)
        _check(lib().tfg_walk_window(self.ctx, int(steps), int(policy),
                                     ctypes.c_void_p(mlp_params.data_ptr()) if mlp_params is not None else None,
                                     ctypes.c_uint32(eps_thresh), ctypes.c_void_p(self._wscratch.data_ptr()),
                                     self._wscratch.numel(),
                                     ctypes.c_void_p(choices.data_ptr()) if choices is not None else None,
                                     ctypes.byref(spec) if spec is not None else None))
        return choices

    walk_window = tfg_walk_window

    def tfg_walk_window_noalloc(self, steps: int, policy: int = 0, mlp_params=None, eps_thresh: int = 0,
                                d_choices=None):
        """tfg_walk_window with the library's own static scratch (no device
        allocation by the call).  d_choices: optional caller-owned int32 device
        tensor [steps, walkers] receiving the chosen window indices."""
        _check(lib().tfg_walk_window_noalloc(
            self.ctx, int(steps), int(policy),
            ctypes.c_void_p(mlp_params.data_ptr()) if mlp_params is not None else None,
            ctypes.c_uint32(eps_thresh), ctypes.c_void_p(d_choices.data_ptr()) if d_choices is not None else None,
            None))

    walk_window_noalloc = tfg_walk_window_noalloc

    def window_buffers(self):
        """Views of the last window step's scratch: window rows (int32 [N, W, 2]:
        descriptor and info words), scores (float32 [N, W]), window sizes (int32 [N]); W = 256."""
        torch, N, W = self.torch, self.total, WINDOW
        b = self._wscratch
        desc = b[: N * W * 8].view(torch.int32).view(N, W, 2)
        score = b[N * W * 8: N * W * 12].view(torch.float32).view(N, W)
        kwin = b[N * W * 12: N * W * 12 + N * 4].view(torch.int32)
        return desc, score, kwin

    def tfg_window_dump(self, features: bool = True):
        """The window of every walker's next window-mode step, without stepping:
        (features bf16 [N, W, 32] or None, rows int32 [N, W, 2], sizes int32 [N])."""
        torch, N, W = self.torch, self.total, WINDOW
        feat = torch.zeros((N, W, 32), dtype=torch.bfloat16, device="cuda") if features else None
        desc = torch.zeros((N, W, 2), dtype=torch.int32, device="cuda")
        kwin = torch.zeros(N, dtype=torch.int32, device="cuda")
        with torch.cuda.stream(self.stream):
            _check(lib().tfg_window_dump(self.ctx, ctypes.c_void_p(feat.data_ptr()) if feat is not None else None,
                                         ctypes.c_void_p(desc.data_ptr()), ctypes.c_void_p(kwin.data_ptr())))
        self.sync()
        return feat, desc, kwin

    window_dump = tfg_window_dump

    def tfg_checkpoint(self) -> bytes:
        used = ctypes.c_size_t()
        _check(lib().tfg_checkpoint(self.ctx, None, 0, ctypes.byref(used)))
        buf = np.zeros(used.value, dtype=np.uint8)
        _check(lib().tfg_checkpoint(self.ctx, _ptr(buf), used.value, ctypes.byref(used)))
        return buf.tobytes()

    checkpoint = tfg_checkpoint

    def tfg_restore(self, data: bytes):
        buf = np.frombuffer(data, dtype=np.uint8).copy()
        _check(lib().tfg_restore(self.ctx, _ptr(buf), buf.size))

    restore = tfg_restore

    def close(self):
        if getattr(self, "ctx", None):
            lib().tfg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
