"""GB300 (sm_103a) tall-skinny QR by randomized CholeskyQR with LU partial
pivoting (RCLUPP, RCLUPPr) plus CholeskyQR2 and LC2 -- Python binding.

The computation lives in ``librclupp.so`` (hand-written CUDA kernels behind
the C ABI of ``include/rclupp.h``).  This module only marshals arguments:
it takes torch CUDA tensors (float64), passes their device pointers,
leading dimensions and the current torch stream to the C entry points of the
same names, and turns status codes into exceptions.  There is no CPU path:
without the compiled library on a CUDA device every call raises.

Matrices are column-major: an m x n tensor with strides (1, ld), ld >= m,
e.g. ``torch.empty((n, m), dtype=torch.float64, device="cuda").t()``.
Row-major inputs are copied to column-major first (``colmajor``).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = [
    "Status", "RclupError", "Opts", "Info", "SKETCH_GAUSSIAN", "SKETCH_SPARSE_SIGN", "SKETCH_SRHT",
    "R0_HOUSEHOLDER", "R0_GIVENS", "rclupp_givens_r",
    "PREC_FP64", "PREC_SKETCH_BF16", "PREC_SKETCH_FP32", "PREC_EMULATED", "PREC_EMULATED_ALL",
    "PREC_SKETCH_DIGITS",
    "load", "library_path", "exported_symbols", "workspace_size", "colmajor", "empty_colmajor", "Handle",
    "rclupp_factor", "rclupp_r_factor", "cholqr2_factor", "lc2_factor", "rcholqr_factor",
    "scholqr3_factor", "ALGO_RCHOLQR", "ALGO_SCHOLQR3",
    "rclupp_sketch", "rclupp_gram", "rclupp_gram_emulated", "rclupp_trsm_emulated",
    "rclupp_trsm_emulated_wellcond", "rclupp_trsm_gram", "rclupp_cholesky", "rclupp_trmm_upper",
    "rclupp_tall_lupp", "rclupp_sketch_precond", "rclupp_householder_r", "rclupp_gram_noalloc",
    "rclupp_factor_batched", "rclupp_factor_batched_async", "rclupp_set_batch_branches",
    "rclupp_autotune_batched",
    "rclupp_set_batch_policy", "rclupp_get_batch_policy",
    "ALGO_RCLUPP", "ALGO_RCLUPPR",
    "ALGO_CHOLQR2", "ALGO_LC2",
    "profile_enable", "profile_reset", "profile_read", "kernel_launches", "KERNEL_CLASSES", "fp64_peak",
]

SKETCH_GAUSSIAN, SKETCH_SPARSE_SIGN, SKETCH_SRHT = 0, 1, 2
R0_HOUSEHOLDER, R0_GIVENS = 0, 1
PREC_FP64, PREC_SKETCH_BF16, PREC_SKETCH_FP32, PREC_EMULATED, PREC_EMULATED_ALL = 0, 1, 2, 3, 4
PREC_SKETCH_DIGITS = 5


class Status:
    OK = 0
    ERR_ARG = -1
    ERR_CHOL_BREAKDOWN = -2
    ERR_LU_ZERO_PIVOT = -3
    ERR_NONFINITE = -4
    ERR_CUDA = -5
    ERR_TIMEOUT = -6
    ERR_NOMEM = -7
    ERR_UNSUPPORTED = -8


class Opts(ctypes.Structure):
    """rclupp_opts_t: sketch kind, zeta, s, seed, precision, optional explicit S."""
    _fields_ = [("kind", ctypes.c_int32), ("zeta", ctypes.c_int32), ("s", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("prec", ctypes.c_int32), ("order_log2", ctypes.c_int32),
                ("S", ctypes.c_void_p), ("lds", ctypes.c_int64), ("r0_method", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Info(ctypes.Structure):
    """rclupp_info_t: status, failed step, failing column, sketch tier used,
    whether the first pass's Gram ran on the emulated path."""
    _fields_ = [("status", ctypes.c_int32), ("failed_step", ctypes.c_int32), ("info", ctypes.c_int64),
                ("prec_used", ctypes.c_int32), ("emulated", ctypes.c_int32)]


class RclupError(RuntimeError):
    def __init__(self, fn: str, status: int, info: "Info | None" = None):
        msg = "%s: %s (status %d)" % (fn, _status_string(status), status)
        if info is not None and info.failed_step:
            msg += ", step %d, column %d" % (info.failed_step, info.info)
        super().__init__(msg)
        self.status = status
        self.info = info


# ------------------------------------------------------------------ loading

_lock = threading.Lock()
_lib = None

_P, _I64, _I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
_SIGNATURES = {
    "rclupp_create": ([ctypes.POINTER(_P), _P], _I32),
    "rclupp_destroy": ([_P], _I32),
    "rclupp_set_stream": ([_P, _P], _I32),
    "rclupp_workspace_bytes": ([_P, ctypes.POINTER(ctypes.c_size_t)], _I32),
    "rclupp_status_string": ([_I32], ctypes.c_char_p),
    "rclupp_factor": ([_P, _I64, _I64, _P, _I64, ctypes.POINTER(Opts), _P, _I64, _P, _I64,
                       ctypes.POINTER(Info)], _I32),
    "rclupp_r_factor": ([_P, _I64, _I64, _P, _I64, ctypes.POINTER(Opts), _P, _I64, _P, _I64,
                         ctypes.POINTER(Info)], _I32),
    "cholqr2_factor": ([_P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, ctypes.POINTER(Info)], _I32),
    "lc2_factor": ([_P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, ctypes.POINTER(Info)], _I32),
    "rcholqr_factor": ([_P, _I64, _I64, _P, _I64, ctypes.POINTER(Opts), _P, _I64, _P, _I64,
                        ctypes.POINTER(Info)], _I32),
    "scholqr3_factor": ([_P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, ctypes.POINTER(Info)], _I32),
    "rclupp_sketch": ([_P, _I64, _I64, _P, _I64, _I32, ctypes.POINTER(Opts), _P, _I64], _I32),
    "rclupp_gram": ([_P, _I64, _I64, _P, _I64, _I32, _P, _I64], _I32),
    "rclupp_gram_emulated": ([_P, _I64, _I64, _P, _I64, _P, _I64], _I32),
    "rclupp_sketch_rows": ([_P, _I64, _I64, _P, _I64, _I64, _I32, _P, _P, _I64], _I32),
    "rclupp_workspace_size": ([_I32, _I64, _I64, _P, _I32, _P], _I32),
    "rclupp_trsm_emulated": ([_P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64], _I32),
    "rclupp_trsm_emulated_wellcond": ([_P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64,
                                       ctypes.POINTER(ctypes.c_int32)], _I32),
    "rclupp_trsm_gram": ([_P, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64], _I32),
    "rclupp_cholesky": ([_P, _I64, _P, _I64, _P, _I64, ctypes.POINTER(ctypes.c_int64)], _I32),
    "rclupp_trmm_upper": ([_P, _I64, _P, _I64, _P, _I64, _P, _I64], _I32),
    "rclupp_tall_lupp": ([_P, _I64, _I64, _P, _I64, _P, ctypes.POINTER(ctypes.c_int64)], _I32),
    "rclupp_sketch_precond": ([_P, _I64, _I64, _P, _I64, _P, _I64], _I32),
    "rclupp_householder_r": ([_P, _I64, _I64, _P, _I64, _P, _I64], _I32),
    "rclupp_givens_r": ([_P, _I64, _I64, _P, _I64, _P, _I64], _I32),
    "rclupp_set_batch_policy": ([_P, _I32, _I32], _I32),
    "rclupp_get_batch_policy": ([_P, _P, _P, _P], _I32),
    "rclupp_sketch_precond_r0": ([_P, _I64, _I64, _P, _I64, _I32, _P, _I64], _I32),
    "rclupp_gram_noalloc": ([_I64, _I64, _P, _I64, _P, _I64, _P], _I32),
    "rclupp_factor_batched": ([_P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], _I32),
    "rclupp_factor_batched_async": ([_P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P], _I32),
    "rclupp_set_batch_branches": ([_P, _I32], _I32),
    "rclupp_autotune_batched": ([_P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                 ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)], _I32),
    "rclupp_profile_enable": ([ctypes.c_int], None),
    "rclupp_profile_reset": ([], None),
    "rclupp_profile_get": ([ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_char_p)], _I32),
    "rclupp_kernel_launches": ([], ctypes.c_ulonglong),
    "rclupp_set_wait_limit": ([_P, ctypes.c_uint64], _I32),
    "rclupp_inject_fault": ([_P, _I32], _I32),
    "rclupp_profile_fp64_peak": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)], _I32),
}

KERNEL_CLASSES = ["sketch_gauss", "sketch_sparse", "gram", "trsm_gram", "trsm", "reduce", "lu_col",
                  "lu_trailing", "lu_u12", "small_precond", "cholesky", "trmm", "pad", "sketch_tc",
                  "gram_emu", "emu_aux", "trsm_emu", "sketch_srht", "fp64_peak"]


def profile_enable(on: bool = True) -> None:
    """Time every kernel launch with CUDA events on its stream (benchmarks)."""
    load().rclupp_profile_enable(1 if on else 0)


def profile_reset() -> None:
    load().rclupp_profile_reset()


def profile_read() -> dict:
    """{class name: (timed launches, total ms)} for every kernel class."""
    lib = load()
    out = {}
    for kid in range(len(KERNEL_CLASSES)):
        n = ctypes.c_longlong(0)
        ms = ctypes.c_double(0.0)
        name = ctypes.c_char_p()
        lib.rclupp_profile_get(kid, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(name))
        out[name.value.decode()] = (int(n.value), float(ms.value))
    return out


def fp64_peak(stream=None) -> dict:
    """Measured FP64-pipe rate of the current device (DFMA microbenchmark on
    the current torch stream): {"gflops", "ms", "sms", "clock_mhz"}."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    g, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    sms, mhz = ctypes.c_int32(0), ctypes.c_int32(0)
    st = load().rclupp_profile_fp64_peak(ctypes.c_void_p(stream), ctypes.byref(g), ctypes.byref(ms),
                                         ctypes.byref(sms), ctypes.byref(mhz))
    _raise("rclupp_profile_fp64_peak", st)
    return {"gflops": g.value, "ms": ms.value, "sms": int(sms.value), "clock_mhz": int(mhz.value)}


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().rclupp_kernel_launches())


def workspace_size(algo, m, n, *, s=None, kind=SKETCH_GAUSSIAN, zeta=8, prec=PREC_FP64,
                   q_aliases_x=False) -> int:
    """Device workspace bytes one factorization needs (no GPU work)."""
    o = Opts()
    o.kind, o.zeta, o.s, o.seed, o.prec = int(kind), int(zeta), int(s if s is not None else 2 * n), 0, int(prec)
    out = ctypes.c_size_t(0)
    st = load().rclupp_workspace_size(int(algo), int(m), int(n), ctypes.byref(o), int(bool(q_aliases_x)),
                                      ctypes.byref(out))
    _raise("rclupp_workspace_size", st)
    return int(out.value)


def library_path() -> str:
    return _build.LIB


def exported_symbols():
    """Names of the C entry points this binding expects the library to export."""
    return sorted(_SIGNATURES)


def load(build: bool = True):
    """Load librclupp.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            if build:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("librclupp.so is missing; run __graft_entry__.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _status_string(status: int) -> str:
    try:
        return load(build=False).rclupp_status_string(status).decode()
    except Exception:
        return "status"


# ------------------------------------------------------------------ tensors

def _torch():
    import torch
    return torch


def colmajor(t):
    """(tensor, ld) with t column-major (strides (1, ld)); copies when needed."""
    torch = _torch()
    if t.dtype != torch.float64:
        raise TypeError("float64 tensors required")
    if not t.is_cuda:
        raise TypeError("CUDA tensors required (the library has no CPU path)")
    if t.dim() != 2:
        raise ValueError("2-D tensors required")
    m, n = t.shape
    if t.stride(0) == 1 and (n == 1 or t.stride(1) >= max(1, m)):
        return t, max(t.stride(1), max(1, m)) if n > 1 else max(1, m)
    c = t.t().contiguous().t()
    return c, max(1, m)


def empty_colmajor(m: int, n: int, device=None):
    torch = _torch()
    return torch.empty((n, m), dtype=torch.float64, device=device or "cuda").t()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Handle:
    """Owns an rclupp handle (workspace + status buffer) on one device."""

    def __init__(self, device=None):
        torch = _torch()
        self.device = torch.device(device or "cuda", torch.cuda.current_device()) \
            if device is None else torch.device(device)
        self._lib = load()
        h = _P()
        with torch.cuda.device(self.device):
            st = self._lib.rclupp_create(ctypes.byref(h), _P(torch.cuda.current_stream().cuda_stream))
        if st != Status.OK:
            raise RclupError("rclupp_create", st)
        self._h = h

    def bind(self):
        torch = _torch()
        self._lib.rclupp_set_stream(self._h, _P(torch.cuda.current_stream(self.device).cuda_stream))
        return self._h

    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t(0)
        self._lib.rclupp_workspace_bytes(self._h, ctypes.byref(v))
        return int(v.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.rclupp_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# One handle per (host thread, device).  A handle holds one stream binding and
# one workspace that a single call at a time may use, and the C calls run
# without the GIL: threads that shared a handle could rebind its stream under
# each other's call and overlap in its workspace.
_local = threading.local()


def _thread_handles() -> dict:
    d = getattr(_local, "handles", None)
    if d is None:
        d = _local.handles = {}
    return d


def _device_index(device) -> int:
    torch = _torch()
    dev = torch.device("cuda") if device is None else torch.device(device)
    return torch.cuda.current_device() if dev.index is None else int(dev.index)


def _device_handle(device=None) -> Handle:
    """The calling thread's handle on `device` (default: the current device)."""
    idx = _device_index(device)
    handles = _thread_handles()
    h = handles.get(idx)
    if h is None:
        h = handles[idx] = Handle("cuda:%d" % idx)
    return h


def _handle(t) -> Handle:
    return _device_handle(t.device)


def _opts(kind=SKETCH_GAUSSIAN, s=None, zeta=8, seed=0, prec=PREC_FP64, S=None, n=None, order_log2=0,
          r0=R0_HOUSEHOLDER):
    o = Opts()
    o.r0_method = int(r0)
    o.kind = int(kind)
    o.zeta = int(zeta)
    o.s = int(s if s is not None else 2 * n)
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    o.prec = int(prec)
    o.order_log2 = int(order_log2)
    if S is not None:
        S, lds = colmajor(S)
        o.S = S.data_ptr()
        o.lds = lds
    else:
        o.S = None
        o.lds = 0
    return o, S


def _raise(fn, st, info=None, check=True):
    if st != Status.OK and check:
        raise RclupError(fn, st, info)


# -------------------------------------------------------------- drivers

def _factor(fn_name, X, sketch=True, Q=None, R=None, check=True, **kw):
    X, ldx = colmajor(X)
    m, n = X.shape
    Q = empty_colmajor(m, n, X.device) if Q is None else Q
    Q, ldq = colmajor(Q)
    R = empty_colmajor(n, n, X.device) if R is None else R
    R, ldr = colmajor(R)
    h = _handle(X)
    info = Info()
    lib = load()
    if sketch:
        o, S_keep = _opts(n=n, **kw)
        st = getattr(lib, fn_name)(h.bind(), m, n, _ptr(X), ldx, ctypes.byref(o), _ptr(Q), ldq,
                                   _ptr(R), ldr, ctypes.byref(info))
    else:
        st = getattr(lib, fn_name)(h.bind(), m, n, _ptr(X), ldx, _ptr(Q), ldq, _ptr(R), ldr,
                                   ctypes.byref(info))
    _raise(fn_name, st, info, check)
    return Q, R, info


def rclupp_factor(X, *, s=None, kind=SKETCH_GAUSSIAN, zeta=8, seed=0, prec=PREC_FP64, S=None,
                  Q=None, R=None, check=True, r0=R0_HOUSEHOLDER, order_log2=0):
    """[Q, R] = RCLUPP(X) (Algorithm 6).  Returns (Q, R, Info)."""
    return _factor("rclupp_factor", X, True, Q, R, check, s=s, kind=kind, zeta=zeta, seed=seed,
                   prec=prec, S=S, r0=r0, order_log2=order_log2)


def rclupp_r_factor(X, *, s=None, kind=SKETCH_GAUSSIAN, zeta=8, seed=0, prec=PREC_FP64, S=None,
                    Q=None, R=None, check=True, r0=R0_HOUSEHOLDER, order_log2=0):
    """[Q, R] = RCLUPPr(X) (Algorithm 7).  Returns (Q, R, Info)."""
    return _factor("rclupp_r_factor", X, True, Q, R, check, s=s, kind=kind, zeta=zeta, seed=seed,
                   prec=prec, S=S, r0=r0, order_log2=order_log2)


def cholqr2_factor(X, *, Q=None, R=None, check=True):
    """[Q, R] = CholeskyQR2(X) (Algorithm 2).  Returns (Q, R, Info)."""
    return _factor("cholqr2_factor", X, False, Q, R, check)


def lc2_factor(X, *, Q=None, R=None, check=True):
    """[Q, R] = LC2(X) (Algorithm 4).  Returns (Q, R, Info)."""
    return _factor("lc2_factor", X, False, Q, R, check)


def rcholqr_factor(X, *, s=None, kind=SKETCH_GAUSSIAN, zeta=8, seed=0, prec=PREC_FP64, S=None,
                   Q=None, R=None, check=True, r0=R0_HOUSEHOLDER, order_log2=0):
    """[Q, R] = RCholeskyQR(X) (Algorithm 5, one sketch, one CholeskyQR)."""
    return _factor("rcholqr_factor", X, True, Q, R, check, s=s, kind=kind, zeta=zeta, seed=seed,
                   prec=prec, S=S, r0=r0, order_log2=order_log2)


def scholqr3_factor(X, *, Q=None, R=None, check=True):
    """[Q, R] = SCholeskyQR3(X) (Algorithm 3)."""
    return _factor("scholqr3_factor", X, False, Q, R, check)


# ---------------------------------------------------------------- steps

def rclupp_sketch(A, *, s, kind=SKETCH_GAUSSIAN, zeta=8, seed=0, prec=PREC_FP64, S=None,
                  unit_lower=False, Y=None, row0=0, order_log2=0):
    """Y = S A (s x n); with row0 > 0, A is the row block starting at global
    row row0 of a taller matrix and Y its partial sketch.  order_log2: the
    SRHT's Hadamard order 2^b (0: the smallest power of two >= row0 + m)."""
    A, lda = colmajor(A)
    m, n = A.shape
    Y = empty_colmajor(s, n, A.device) if Y is None else Y
    Y, ldy = colmajor(Y)
    o, S_keep = _opts(kind=kind, s=s, zeta=zeta, seed=seed, prec=prec, S=S, n=n, order_log2=order_log2)
    st = load().rclupp_sketch_rows(_handle(A).bind(), m, n, _ptr(A), lda, int(row0),
                                   int(bool(unit_lower)), ctypes.byref(o), _ptr(Y), ldy)
    _raise("rclupp_sketch", st)
    return Y


def rclupp_gram(A, *, unit_lower=False, G=None):
    """G = A^T A."""
    A, lda = colmajor(A)
    m, n = A.shape
    G = empty_colmajor(n, n, A.device) if G is None else G
    G, ldg = colmajor(G)
    st = load().rclupp_gram(_handle(A).bind(), m, n, _ptr(A), lda, int(bool(unit_lower)), _ptr(G),
                            ldg)
    _raise("rclupp_gram", st)
    return G


def rclupp_gram_emulated(A, *, G=None):
    """G = A^T A as binary64-emulating split-bf16 products on the tensor cores."""
    A, lda = colmajor(A)
    m, n = A.shape
    G = empty_colmajor(n, n, A.device) if G is None else G
    G, ldg = colmajor(G)
    st = load().rclupp_gram_emulated(_handle(A).bind(), m, n, _ptr(A), lda, _ptr(G), ldg)
    _raise("rclupp_gram_emulated", st)
    return G


def rclupp_trsm_emulated(A, R, *, Q=None):
    """Q = A R^{-1} with binary64-emulating tensor-core block products."""
    A, lda = colmajor(A)
    m, n = A.shape
    R, ldr = colmajor(R)
    Q = empty_colmajor(m, n, A.device) if Q is None else Q
    Q, ldq = colmajor(Q)
    st = load().rclupp_trsm_emulated(_handle(A).bind(), m, n, _ptr(A), lda, _ptr(R), ldr, _ptr(Q), ldq)
    _raise("rclupp_trsm_emulated", st)
    return Q


def rclupp_trsm_emulated_wellcond(A, R, *, Q=None):
    """Q = A R^{-1} for a well-conditioned R: the emulated product with R^{-1}
    when ||R||_1 ||R^{-1}||_1 <= 100, else the emulated substitution.
    Returns (Q, form) with form 1 for the product, 0 for the substitution."""
    A, lda = colmajor(A)
    m, n = A.shape
    R, ldr = colmajor(R)
    Q = empty_colmajor(m, n, A.device) if Q is None else Q
    Q, ldq = colmajor(Q)
    form = ctypes.c_int32(-1)
    st = load().rclupp_trsm_emulated_wellcond(_handle(A).bind(), m, n, _ptr(A), lda, _ptr(R), ldr, _ptr(Q),
                                              ldq, ctypes.byref(form))
    _raise("rclupp_trsm_emulated_wellcond", st)
    return Q, int(form.value)


ALGO_RCLUPP, ALGO_RCLUPPR, ALGO_CHOLQR2, ALGO_LC2, ALGO_RCHOLQR, ALGO_SCHOLQR3 = 0, 1, 2, 3, 4, 5


def rclupp_factor_batched(Xs, *, algo=ALGO_RCLUPP, s=None, kind=SKETCH_GAUSSIAN, zeta=8, seed=0,
                          Qs=None, Rs=None, check=True, prec=PREC_FP64, r0=R0_HOUSEHOLDER):
    """Factor a list of column-major matrices in one batched call (one CUDA
    graph).  s is a per-problem list (or None for 2 n); seed is a list or an
    int (then seed + i for problem i); prec is PREC_FP64 (binary64 sketch),
    PREC_SKETCH_FP32 (three-term tensor-core sketch), PREC_SKETCH_DIGITS or an
    emulated tier (digit-tier sketch); no escalation inside a graph.
    Returns (Qs, Rs, statuses)."""
    a = _batch_args(Xs, Qs, Rs, s, kind, zeta, seed, prec, r0)
    st = load().rclupp_factor_batched(a["h"], int(algo), a["count"], *a["args"], a["pst"])
    _raise("rclupp_factor_batched", st, None, check)
    return a["Qs"], a["Rs"], a["status"]


def rclupp_factor_batched_async(Xs, *, algo=ALGO_RCLUPP, s=None, kind=SKETCH_GAUSSIAN, zeta=8,
                                seed=0, Qs=None, Rs=None, prec=PREC_FP64, r0=R0_HOUSEHOLDER,
                                d_status=None):
    """The batched call enqueued on the current stream without waiting (it can
    be recorded by a caller's CUDA graph capture): returns (Qs, Rs, d_status),
    d_status an int32 tensor on the device holding each problem's status once
    the stream reaches it.  While capturing, the handle's workspace must
    already fit the batch (an earlier call outside the capture)."""
    torch = _torch()
    a = _batch_args(Xs, Qs, Rs, s, kind, zeta, seed, prec, r0)
    if d_status is None:
        d_status = torch.zeros(a["count"], dtype=torch.int32, device=a["Qs"][0].device)
    st = load().rclupp_factor_batched_async(a["h"], int(algo), a["count"], *a["args"],
                                            _P(d_status.data_ptr()))
    _raise("rclupp_factor_batched_async", st)
    return a["Qs"], a["Rs"], d_status


def rclupp_autotune_batched(Xs, *, algo=ALGO_RCLUPP, s=None, kind=SKETCH_GAUSSIAN, zeta=8, seed=0,
                            Qs=None, Rs=None, prec=PREC_FP64, r0=R0_HOUSEHOLDER):
    """Time the batch over candidate branch counts and keep the fastest in
    the handle.  Returns (branches, ms of one batched call)."""
    a = _batch_args(Xs, Qs, Rs, s, kind, zeta, seed, prec, r0)
    best = ctypes.c_int32(0)
    ms = ctypes.c_float(0.0)
    st = load().rclupp_autotune_batched(a["h"], int(algo), a["count"], *a["args"], ctypes.byref(best),
                                        ctypes.byref(ms))
    _raise("rclupp_autotune_batched", st)
    return int(best.value), float(ms.value)


def _batch_args(Xs, Qs, Rs, s, kind, zeta, seed, prec=0, r0=0):
    import numpy as np
    count = len(Xs)
    Xs = [colmajor(x) for x in Xs]
    dev = Xs[0][0].device
    Qs = [empty_colmajor(x.shape[0], x.shape[1], dev) for x, _ in Xs] if Qs is None else list(Qs)
    Rs = [empty_colmajor(x.shape[1], x.shape[1], dev) for x, _ in Xs] if Rs is None else list(Rs)
    qc = [colmajor(q) for q in Qs]
    rc = [colmajor(r) for r in Rs]
    m = np.array([x.shape[0] for x, _ in Xs], dtype=np.int64)
    n = np.array([x.shape[1] for x, _ in Xs], dtype=np.int64)
    ldx = np.array([ld for _, ld in Xs], dtype=np.int64)
    ldq = np.array([ld for _, ld in qc], dtype=np.int64)
    ldr = np.array([ld for _, ld in rc], dtype=np.int64)
    xp = np.array([x.data_ptr() for x, _ in Xs], dtype=np.uint64)
    qp = np.array([q.data_ptr() for q, _ in qc], dtype=np.uint64)
    rp = np.array([r.data_ptr() for r, _ in rc], dtype=np.uint64)
    opts = (Opts * count)()
    for i in range(count):
        opts[i].kind = int(kind)
        opts[i].zeta = int(zeta)
        opts[i].s = int(s[i] if s is not None else 2 * n[i])
        opts[i].seed = int(seed[i] if isinstance(seed, (list, tuple)) else seed + i)
        opts[i].prec = int(prec)
        opts[i].r0_method = int(r0)
        opts[i].S = None
        opts[i].lds = 0
    status = np.zeros(count, dtype=np.int32)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    h = _handle(Xs[0][0])
    # everything the pointers above refer to stays referenced until the call
    # returns, the column-major copies of inputs given in another layout too
    keep = (m, n, xp, ldx, opts, qp, ldq, rp, ldr, status, [x for x, _ in Xs])
    return {"h": h.bind(), "count": count, "keep": keep, "status": status, "pst": p(status),
            "args": (p(m), p(n), p(xp), p(ldx), ctypes.cast(opts, _P), p(qp), p(ldq), p(rp), p(ldr)),
            "Qs": [q for q, _ in qc], "Rs": [r for r, _ in rc]}


def rclupp_set_batch_branches(branches: int, device=None):
    """Parallel branches of the batched graph on the calling thread's handle."""
    st = load().rclupp_set_batch_branches(_device_handle(device)._h, int(branches))
    _raise("rclupp_set_batch_branches", st)


def rclupp_set_batch_policy(grid_div: int = 1, fine_tiles: bool = False, device=None):
    """Launch shapes inside the batched graph (calling thread's handle): CTA-budget
    divisor and finer row tiles."""
    st = load().rclupp_set_batch_policy(_device_handle(device)._h, int(grid_div), int(bool(fine_tiles)))
    _raise("rclupp_set_batch_policy", st)


def rclupp_get_batch_policy(device=None):
    """(branches, grid_div, fine_tiles) of the handle's batched form."""
    b, g, f = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    st = load().rclupp_get_batch_policy(_device_handle(device)._h, ctypes.byref(b), ctypes.byref(g),
                                        ctypes.byref(f))
    _raise("rclupp_get_batch_policy", st)
    return int(b.value), int(g.value), int(f.value)


def rclupp_gram_noalloc(A, *, G=None):
    """G = A^T A through the allocation-free entry point (n <= 128).

    For callers that must not let the library allocate device memory: the
    scratch lives in a fixed array inside the library; no handle is used.
    Calls on one device must not overlap on the GPU (they share that array).
    """
    torch = _torch()
    A, lda = colmajor(A)
    m, n = A.shape
    G = empty_colmajor(n, n, A.device) if G is None else G
    G, ldg = colmajor(G)
    with torch.cuda.device(A.device):
        stream = torch.cuda.current_stream(A.device).cuda_stream
        st = load().rclupp_gram_noalloc(m, n, _ptr(A), lda, _ptr(G), ldg, _P(stream))
    _raise("rclupp_gram_noalloc", st)
    return G


def rclupp_trsm_gram(A, R, *, Q=None, gram=True):
    """Q = A R^{-1} and (when gram) G = Q^T Q.  Returns (Q, G or None)."""
    A, lda = colmajor(A)
    R, ldr = colmajor(R)
    m, n = A.shape
    Q = empty_colmajor(m, n, A.device) if Q is None else Q
    Q, ldq = colmajor(Q)
    G = empty_colmajor(n, n, A.device) if gram else None
    ldg = colmajor(G)[1] if gram else 1
    st = load().rclupp_trsm_gram(_handle(A).bind(), m, n, _ptr(A), lda, _ptr(R), ldr, _ptr(Q), ldq,
                                 _ptr(G), ldg)
    _raise("rclupp_trsm_gram", st)
    return Q, G


def rclupp_cholesky(G, *, check=True):
    """Upper R with G = R^T R.  Returns (R, status, column)."""
    G, ldg = colmajor(G)
    n = G.shape[0]
    R = empty_colmajor(n, n, G.device)
    col = ctypes.c_int64(-1)
    st = load().rclupp_cholesky(_handle(G).bind(), n, _ptr(G), ldg, _ptr(R), n, ctypes.byref(col))
    _raise("rclupp_cholesky", st, None, check)
    return R, st, int(col.value)


def rclupp_trmm_upper(A, B):
    """C = triu(A) triu(B)."""
    A, lda = colmajor(A)
    B, ldb = colmajor(B)
    n = A.shape[0]
    C = empty_colmajor(n, n, A.device)
    st = load().rclupp_trmm_upper(_handle(A).bind(), n, _ptr(A), lda, _ptr(B), ldb, _ptr(C), n)
    _raise("rclupp_trmm_upper", st)
    return C


def rclupp_tall_lupp(A, *, check=True):
    """In-place tall LU with partial pivoting on a column-major copy of A.
    Returns (LU, ipiv (int32, device), status, column)."""
    torch = _torch()
    A, lda = colmajor(A)
    LU = A.clone(memory_format=torch.preserve_format)
    LU, ldl = colmajor(LU)
    m, n = LU.shape
    ipiv = torch.zeros(n, dtype=torch.int32, device=A.device)
    col = ctypes.c_int64(-1)
    st = load().rclupp_tall_lupp(_handle(A).bind(), m, n, _ptr(LU), ldl, _ptr(ipiv), ctypes.byref(col))
    _raise("rclupp_tall_lupp", st, None, check)
    return LU, ipiv, st, int(col.value)


def rclupp_sketch_precond(Y, r0=R0_HOUSEHOLDER):
    """R1 from a sketched matrix (the preconditioner of Algorithm 6, signs normalised),
    R0 by Householder (default) or Givens rotations."""
    Y, ldy = colmajor(Y)
    s, n = Y.shape
    R1 = empty_colmajor(n, n, Y.device)
    if r0 == R0_HOUSEHOLDER:
        st = load().rclupp_sketch_precond(_handle(Y).bind(), s, n, _ptr(Y), ldy, _ptr(R1), n)
    else:
        st = load().rclupp_sketch_precond_r0(_handle(Y).bind(), s, n, _ptr(Y), ldy, int(r0), _ptr(R1), n)
    _raise("rclupp_sketch_precond", st)
    return R1


def rclupp_givens_r(A):
    """R-factor of A by Givens rotations (non-negative diagonal)."""
    A, lda = colmajor(A)
    s, n = A.shape
    R = empty_colmajor(n, n, A.device)
    st = load().rclupp_givens_r(_handle(A).bind(), s, n, _ptr(A), lda, _ptr(R), n)
    _raise("rclupp_givens_r", st)
    return R


def rclupp_householder_r(A):
    """R-factor of the Householder QR of A (LAPACK larfg convention)."""
    A, lda = colmajor(A)
    s, n = A.shape
    R = empty_colmajor(n, n, A.device)
    st = load().rclupp_householder_r(_handle(A).bind(), s, n, _ptr(A), lda, _ptr(R), n)
    _raise("rclupp_householder_r", st)
    return R
