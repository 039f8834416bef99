"""CPU oracle for the tall-skinny QR path (test infrastructure, not product).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  It wraps ``rclupp_oracle.c``: a plain,
sequential-sum FP64 implementation of CholeskyQR, CholeskyQR2 (Algorithm 2),
LC2 (Algorithm 4), RCLUPP (Algorithm 6) and RCLUPPr (Algorithm 7), plus the
building blocks they are made of and the generated sketches (Gaussian,
sparse-sign, subsampled randomized Hadamard), compiled with gcc
``-ffp-contract=off``.

All matrix arguments are numpy float64 arrays; results are returned
column-major (Fortran order).  Status codes: 0 ok, -1 bad argument,
-2 Cholesky breakdown, -3 zero LU pivot, -7 out of memory.

Parity pins: every routine is checked against values the paper or plain
mathematics fix (closed forms, uniqueness of the positive-diagonal QR,
brute force in extended precision, the paper's error bounds), in
``tests/test_oracle_pins.py`` and ``tests/test_oracle_srht.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rclupp_oracle.c")
_LIB = os.path.join(_HERE, "librclupp_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, CHOL_BREAKDOWN, LU_ZERO_PIVOT, ERR_NOMEM = 0, -1, -2, -3, -7
SKETCH_DENSE, SKETCH_SPARSE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = base + ["-fopenmp", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:  # toolchain without OpenMP: build single-threaded
        r = subprocess.run(base + [_SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P, I64, I32, U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
            sig = {
                "orc_num_threads": ([], I32),
                "orc_set_num_threads": ([I32], None),
                "orc_gram": ([I64, I64, P, I64, P, I64], None),
                "orc_cholesky": ([I64, P, I64, P, I64, P], I32),
                "orc_trsm_right_upper": ([I64, I64, P, I64, P, I64, P, I64], None),
                "orc_trmm_upper": ([I64, P, I64, P, I64, P, I64], None),
                "orc_gepp": ([I64, I64, P, I64, P, P], I32),
                "orc_householder_r": ([I64, I64, P, I64, P, I64], None),
                "orc_givens_r": ([I64, I64, P, I64, P, I64], None),
                "orc_sketch_dense": ([I64, I64, I64, P, I64, P, I64, P, I64], None),
                "orc_sketch_sparse": ([I64, I64, I64, I32, P, P, P, I64, P, I64], None),
                "orc_sketch_precond": ([I64, I64, P, I64, P, I64, P, I32], I32),
                "orc_cholqr": ([I64, I64, P, I64, P, I64, P, I64, P], I32),
                "orc_cholqr2": ([I64, I64, P, I64, P, I64, P, I64, P], I32),
                "orc_lc2": ([I64, I64, P, I64, P, I64, P, I64, P], I32),
                "orc_rclupp": ([I64, I64, P, I64, I32, I64, I32, P, I64, P, P, P, I64, P, I64, P, I32], I32),
                "orc_rcluppr": ([I64, I64, P, I64, I32, I64, I32, P, I64, P, P, P, I64, P, I64, P, I32], I32),
                "orc_rcluppr_precond": ([I64, I64, P, I64, I32, I64, I32, P, I64, P, P, P, I64, P, I32], I32),
                "orc_philox4x32_10": ([P, P, P], None),
                "orc_ln_f32": ([ctypes.c_float], ctypes.c_float),
                "orc_cossin_2pi_f32": ([ctypes.c_float, P, P], None),
                "orc_gauss_entry": ([U64, I64, I64], ctypes.c_float),
                "orc_gaussian_sketch_matrix": ([I64, I64, U64, P, I64], None),
                "orc_sparse_sign_column": ([U64, I64, I64, I32, P, P], None),
                "orc_sparse_sign_pattern": ([I64, I64, I32, U64, P, P], None),
                "orc_rcholqr": ([I64, I64, P, I64, I32, I64, I32, P, I64, P, P, P, I64, P, I64, P, I32], I32),
                "orc_scholqr3": ([I64, I64, P, I64, P, I64, P, I64, P], I32),
                "orc_scholqr3_shift": ([I64, I64, P, I64], ctypes.c_double),
                "orc_round_bf16": ([ctypes.c_double], ctypes.c_double),
                "orc_sketch_bf16": ([I64, I64, I64, U64, I32, P, I64, P, I64], I32),
                "orc_normal_quantile": ([ctypes.c_double], ctypes.c_double),
                "orc_tier_levels": ([P], None),
                "orc_tier_sketch_entries": ([I64, I64, U64, P, I64], I32),
                "orc_sketch_digits": ([I64, I64, I64, U64, P, I64, P, I64], I32),
                "orc_srht_perm_one": ([I32, U64, I64], I64),
                "orc_srht_perm": ([I32, I64, U64, P], None),
                "orc_srht_signs": ([U64, I64, I64, P], None),
                "orc_srht_dense": ([I64, I64, I64, I64, P, P, P, I64], None),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _f(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def set_num_threads(k: int) -> None:
    """Threads the oracle's OpenMP loops use from now on (timing only)."""
    _load().orc_set_num_threads(int(k))


def num_threads() -> int:
    return int(_load().orc_num_threads())


class OracleError(RuntimeError):
    def __init__(self, status: int, info: int):
        super().__init__("oracle status %d (info %d)" % (status, info))
        self.status, self.info = status, info


def _check(st: int, info: np.ndarray, raise_on_error: bool):
    if st != OK and raise_on_error:
        raise OracleError(st, int(info[0]))
    return st


# ---------------------------------------------------------------- blocks ---

def gram(x) -> np.ndarray:
    """G = X^T X (the Gram product of Algorithm 1)."""
    x = _f(x)
    m, n = x.shape
    g = np.zeros((n, n), order="F")
    _load().orc_gram(m, n, _p(x), m, _p(g), n)
    return g


def cholesky(g, raise_on_error: bool = True):
    """Upper R with G = R^T R (the Cholesky factorization of Algorithm 1).
    Returns (R, status, info)."""
    g = _f(g)
    n = g.shape[0]
    r = np.zeros((n, n), order="F")
    info = np.zeros(1, dtype=np.int64)
    st = _load().orc_cholesky(n, _p(g), n, _p(r), n, _p(info))
    _check(st, info, raise_on_error)
    return r, st, int(info[0])


def trsm(x, r) -> np.ndarray:
    """Q = X R^{-1} by row-wise substitution (the solve of Algorithm 1)."""
    x, r = _f(x), _f(r)
    m, n = x.shape
    q = np.zeros((m, n), order="F")
    _load().orc_trsm_right_upper(m, n, _p(x), m, _p(r), n, _p(q), m)
    return q


def trmm_upper(a, b) -> np.ndarray:
    """C = A B for upper-triangular A, B."""
    a, b = _f(a), _f(b)
    n = a.shape[0]
    c = np.zeros((n, n), order="F")
    _load().orc_trmm_upper(n, _p(a), n, _p(b), n, _p(c), n)
    return c


def gepp(a, raise_on_error: bool = True):
    """In-place-style GEPP: returns (LU, ipiv, status, info); LU holds M below
    the diagonal (unit diagonal implied) and N on and above it."""
    lu = _f(a).copy(order="F")
    m, n = lu.shape
    ipiv = np.zeros(min(m, n), dtype=np.int32)
    info = np.zeros(1, dtype=np.int64)
    st = _load().orc_gepp(m, n, _p(lu), m, _p(ipiv), _p(info))
    _check(st, info, raise_on_error)
    return lu, ipiv, st, int(info[0])


def unit_lower(lu) -> np.ndarray:
    m, n = lu.shape
    out = np.tril(lu, -1)[:, :n].copy(order="F")
    out[np.arange(n), np.arange(n)] = 1.0
    return out


def upper(lu) -> np.ndarray:
    n = lu.shape[1]
    return np.triu(lu[:n, :n]).copy(order="F")


def householder_r(a) -> np.ndarray:
    """R-factor of the thin Householder QR (LAPACK larfg sign convention)."""
    a = _f(a)
    s, n = a.shape
    r = np.zeros((n, n), order="F")
    _load().orc_householder_r(s, n, _p(a), s, _p(r), n)
    return r


def sketch_dense(S, x) -> np.ndarray:
    """Y = S X with an explicit dense S."""
    S, x = _f(S), _f(x)
    s, m = S.shape
    n = x.shape[1]
    y = np.zeros((s, n), order="F")
    _load().orc_sketch_dense(s, m, n, _p(S), s, _p(x), m, _p(y), s)
    return y


def sketch_sparse(s: int, zeta: int, rows, signs, x) -> np.ndarray:
    """Y = S X with S given by its per-column rows and signs (+-1/sqrt(zeta))."""
    x = _f(x)
    m, n = x.shape
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    signs = np.ascontiguousarray(signs, dtype=np.int8)
    y = np.zeros((s, n), order="F")
    _load().orc_sketch_sparse(s, m, n, zeta, _p(rows), _p(signs), _p(x), m, _p(y), s)
    return y


R0_METHODS = {"householder": 0, "givens": 1}


def givens_r(a) -> np.ndarray:
    """R-factor of A (s x n) by Givens rotations, bottom-up per column."""
    a = _f(a)
    s, n = a.shape
    r = np.zeros((n, n), order="F")
    _load().orc_givens_r(s, n, _p(a), s, _p(r), n)
    return r


def sketch_precond(y, raise_on_error: bool = True, r0: str = "householder"):
    """R1 from the sketched matrix (the preconditioner of Algorithm 6 + sign fix), R0 by
    Householder (the paper's choice) or Givens rotations. Returns (R1, status, info)."""
    y = _f(y)
    s, n = y.shape
    r1 = np.zeros((n, n), order="F")
    info = np.zeros(1, dtype=np.int64)
    st = _load().orc_sketch_precond(s, n, _p(y), s, _p(r1), n, _p(info), R0_METHODS[r0])
    _check(st, info, raise_on_error)
    return r1, st, int(info[0])


def rcluppr_precond(x, S=None, sparse=None, raise_on_error: bool = True, r0: str = "householder"):
    """R1 of RCLUPPr (the preconditioner of Algorithm 7): [M, N, P] = LU(X),
    R0 = R-factor of S M, R1 = R0 N, signs normalised; dense S or
    sparse=(s, zeta, rows, signs). Returns (R1, status, info)."""
    x = _f(x)
    m, n = x.shape
    r1 = np.zeros((n, n), order="F")
    info = np.zeros(1, dtype=np.int64)
    lib = _load()
    if sparse is not None:
        s, zeta, rows, signs = sparse
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        signs = np.ascontiguousarray(signs, dtype=np.int8)
        st = lib.orc_rcluppr_precond(m, n, _p(x), m, SKETCH_SPARSE, s, zeta, None, 0, _p(rows), _p(signs),
                                     _p(r1), n, _p(info), R0_METHODS[r0])
    else:
        S = _f(S)
        st = lib.orc_rcluppr_precond(m, n, _p(x), m, SKETCH_DENSE, S.shape[0], 0, _p(S), S.shape[0], None,
                                     None, _p(r1), n, _p(info), R0_METHODS[r0])
    _check(st, info, raise_on_error)
    return r1, st, int(info[0])


# -------------------------------------------------------------- drivers ---

def _qr_out(m, n):
    return np.zeros((m, n), order="F"), np.zeros((n, n), order="F"), np.zeros(1, dtype=np.int64)


def cholqr(x, raise_on_error: bool = True):
    x = _f(x)
    m, n = x.shape
    q, r, info = _qr_out(m, n)
    st = _load().orc_cholqr(m, n, _p(x), m, _p(q), m, _p(r), n, _p(info))
    _check(st, info, raise_on_error)
    return q, r, st


def cholqr2(x, raise_on_error: bool = True):
    """[Q, R] = CholeskyQR2(X) (Algorithm 2). Returns (Q, R, status)."""
    x = _f(x)
    m, n = x.shape
    q, r, info = _qr_out(m, n)
    st = _load().orc_cholqr2(m, n, _p(x), m, _p(q), m, _p(r), n, _p(info))
    _check(st, info, raise_on_error)
    return q, r, st


def lc2(x, raise_on_error: bool = True):
    """[Q, R] = LC2(X) (Algorithm 4). Returns (Q, R, status)."""
    x = _f(x)
    m, n = x.shape
    q, r, info = _qr_out(m, n)
    st = _load().orc_lc2(m, n, _p(x), m, _p(q), m, _p(r), n, _p(info))
    _check(st, info, raise_on_error)
    return q, r, st


def _rand_driver(fn, x, S=None, sparse=None, raise_on_error=True, r0="householder"):
    x = _f(x)
    m, n = x.shape
    q, r, info = _qr_out(m, n)
    lib = _load()
    if sparse is not None:
        s, zeta, rows, signs = sparse
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        signs = np.ascontiguousarray(signs, dtype=np.int8)
        st = getattr(lib, fn)(m, n, _p(x), m, SKETCH_SPARSE, s, zeta, None, 0, _p(rows), _p(signs),
                              _p(q), m, _p(r), n, _p(info), R0_METHODS[r0])
    else:
        S = _f(S)
        s = S.shape[0]
        st = getattr(lib, fn)(m, n, _p(x), m, SKETCH_DENSE, s, 0, _p(S), s, None, None,
                              _p(q), m, _p(r), n, _p(info), R0_METHODS[r0])
    _check(st, info, raise_on_error)
    return q, r, st


def rclupp(x, S=None, sparse=None, raise_on_error: bool = True, r0: str = "householder"):
    """[Q, R] = RCLUPP(X) (Algorithm 6) with dense S or sparse=(s, zeta, rows, signs);
    r0 = "householder" (the paper's choice) or "givens" for the R-factor R0."""
    return _rand_driver("orc_rclupp", x, S, sparse, raise_on_error, r0)


def rcluppr(x, S=None, sparse=None, raise_on_error: bool = True, r0: str = "householder"):
    """[Q, R] = RCLUPPr(X) (Algorithm 7) with dense S or sparse=(s, zeta, rows, signs)."""
    return _rand_driver("orc_rcluppr", x, S, sparse, raise_on_error, r0)


def rcholqr(x, S=None, sparse=None, raise_on_error: bool = True, r0: str = "householder"):
    """[Q, R] = RCholeskyQR(X) (Algorithm 5, one sketch, one CholeskyQR)."""
    return _rand_driver("orc_rcholqr", x, S, sparse, raise_on_error, r0)


def scholqr3(x, raise_on_error: bool = True):
    """[Q, R] = SCholeskyQR3(X) (Algorithm 3, shift 11(mnu + n(n+1)u)||X||_g^2)."""
    x = _f(x)
    m, n = x.shape
    q, r, info = _qr_out(m, n)
    st = _load().orc_scholqr3(m, n, _p(x), m, _p(q), m, _p(r), n, _p(info))
    _check(st, info, raise_on_error)
    return q, r, st


def scholqr3_shift(m: int, g) -> float:
    """The shift s of SCholeskyQR3 from the Gram matrix G of an m-row X."""
    g = _f(g)
    n = g.shape[0]
    return float(_load().orc_scholqr3_shift(m, n, _p(g), n))


# ------------------------------------------------------------ generators ---

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def ln_f32(x: float) -> float:
    return float(_load().orc_ln_f32(ctypes.c_float(x)))


def cossin_2pi_f32(u: float):
    c = np.zeros(1, dtype=np.float32)
    s = np.zeros(1, dtype=np.float32)
    _load().orc_cossin_2pi_f32(ctypes.c_float(u), _p(c), _p(s))
    return float(c[0]), float(s[0])


def gauss_entry(seed: int, r: int, i: int) -> float:
    return float(_load().orc_gauss_entry(seed, r, i))


def gaussian_sketch_matrix(s: int, m: int, seed: int) -> np.ndarray:
    """The on-the-fly Gaussian sketch S (s x m) for ``seed``, materialised."""
    S = np.zeros((s, m), order="F")
    _load().orc_gaussian_sketch_matrix(s, m, seed, _p(S), s)
    return S


def sparse_sign_pattern(s: int, m: int, zeta: int, seed: int):
    """(rows, signs), each of length m*zeta, of the on-the-fly sparse-sign sketch."""
    rows = np.zeros(m * zeta, dtype=np.int32)
    signs = np.zeros(m * zeta, dtype=np.int8)
    _load().orc_sparse_sign_pattern(s, m, zeta, seed, _p(rows), _p(signs))
    return rows, signs


def sparse_to_dense(s: int, m: int, zeta: int, rows, signs) -> np.ndarray:
    S = np.zeros((s, m), order="F")
    val = 1.0 / np.sqrt(zeta)
    cols = np.repeat(np.arange(m), zeta)
    S[np.asarray(rows), cols] = np.where(np.asarray(signs) > 0, val, -val)
    return S


def srht_order_log2(m: int) -> int:
    """b of the SRHT's padded order m' = 2^b: the smallest b with 2^b >= m."""
    b = 0
    while (1 << b) < m:
        b += 1
    return b


def srht_perm(s: int, b: int, seed: int) -> np.ndarray:
    """Sampled rows p_0 .. p_{s-1} of the order-2^b Hadamard matrix (s <= 2^b)."""
    p = np.zeros(s, dtype=np.int64)
    _load().orc_srht_perm(b, s, seed, _p(p))
    return p


def srht_signs(m: int, seed: int, row0: int = 0) -> np.ndarray:
    """Signs d_{row0} .. d_{row0 + m - 1} (int8, +1 or -1)."""
    d = np.zeros(m, dtype=np.int8)
    _load().orc_srht_signs(seed, row0, m, _p(d))
    return d


def srht_dense(s: int, m: int, seed: int, b: int = None, row0: int = 0) -> np.ndarray:
    """Columns row0 .. row0 + m - 1 of the SRHT sketch S = R H D / sqrt(s)
    (s x m, Fortran order); b defaults to srht_order_log2(row0 + m)."""
    return srht_dense_rows(np.arange(s), s, m, seed, b, row0)


def srht_dense_rows(rows, s: int, m: int, seed: int, b: int = None, row0: int = 0) -> np.ndarray:
    """Rows `rows` (indices into 0 .. s-1) of the s-row SRHT sketch, columns
    row0 .. row0 + m - 1 (len(rows) x m, Fortran order)."""
    b = srht_order_log2(row0 + m) if b is None else b
    p = np.ascontiguousarray(srht_perm(s, b, seed)[np.asarray(rows, dtype=np.int64)])
    d = srht_signs(m, seed, row0)
    k = len(p)
    S = np.zeros((k, m), order="F")
    _load().orc_srht_dense(k, s, m, row0, _p(p), _p(d), _p(S), k)
    return S


def round_bf16(x: float) -> float:
    """Nearest bf16 value (8 significant bits, ties to even) of a binary64 value."""
    return float(_load().orc_round_bf16(float(x)))


def normal_quantile(p: float) -> float:
    """Phi^{-1}(p) of the standard normal (bisection on erfc)."""
    return float(_load().orc_normal_quantile(float(p)))


def tier_levels() -> np.ndarray:
    """The tensor-core tiers' 4096 levels T[j] = round(32 Phi^{-1}((j + 1/2) / 4096)) / 32."""
    t = np.zeros(4096)
    _load().orc_tier_levels(_p(t))
    return t


def tier_sketch_z(s: int, m: int, seed: int) -> np.ndarray:
    """Unscaled sketch z_b of the tensor-core tiers (s x m); the sketch is z_b / sqrt(s)."""
    z = np.zeros((s, m), order="F")
    st = _load().orc_tier_sketch_entries(s, m, seed, _p(z), s)
    if st != OK:
        raise OracleError(st, -1)
    return z


def sketch_digits(s: int, seed: int, x) -> np.ndarray:
    """Y = z_b X~ / sqrt(s) with X~ the six-digit (48-bit, per-column exponent)
    rounding of X, the integer sum taken exactly: the digit tier's definition."""
    x = _f(x)
    m, n = x.shape
    y = np.zeros((s, n), order="F")
    st = _load().orc_sketch_digits(s, m, n, seed, _p(x), m, _p(y), s)
    if st != OK:
        raise OracleError(st, -1)
    return y


def sketch_bf16(s: int, seed: int, nterms: int, x) -> np.ndarray:
    """Y = z_b X_split / sqrt(s): the tensor-core tier's sketch definition
    (S entries z_b(r, i) on the grid of the discretised normal; X in one or
    three bf16 terms)."""
    x = _f(x)
    m, n = x.shape
    y = np.zeros((s, n), order="F")
    st = _load().orc_sketch_bf16(s, m, n, seed, nterms, _p(x), m, _p(y), s)
    if st != OK:
        raise OracleError(st, -1)
    return y


def bf16_split(x, nterms: int = 3) -> np.ndarray:
    """Sum of the nterms bf16 terms of each entry (elementwise, via round_bf16)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.vectorize(round_bf16)
    x1 = r(x)
    if nterms == 1:
        return x1
    x2 = r(x - x1)
    x3 = r(x - x1 - x2)
    return x1 + x2 + x3


# ---------------------------------------------------------------- metrics ---

def orthogonality(q) -> float:
    """||Q^T Q - I||_F (the paper's orthogonality measure, Section 5)."""
    q = np.asarray(q, dtype=np.float64)
    n = q.shape[1]
    return float(np.linalg.norm(q.T @ q - np.eye(n), "fro"))


def residual(x, q, r) -> float:
    """||Q R - X||_F / ||X||_F."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(q) @ np.asarray(r) - x, "fro") / np.linalg.norm(x, "fro"))
