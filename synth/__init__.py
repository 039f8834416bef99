"""Seeded synthetic inputs for the tall-skinny QR path (test and bench fixtures).

This module builds input matrices only.  It holds none of the factorization's
arithmetic: orthonormal bases come from ``numpy.linalg.qr`` (LAPACK), and the
explicit sketch matrices are plain draws from numpy's Philox generator.  Both
the CPU oracle and the CUDA library consume what it returns; neither is
imported here.

Matrices are returned column-major (``order='F'``) float64, the layout of the
C-ABI (element (i, j) at ``X[i + j*ld]``).

Constructions follow the paper's experiments (Section 5):
  * ``svd_matrix``       -- X = U diag(sigma) V^T with sigma geometric from 1
                            to 1/kappa, so ||X||_2 = 1 and kappa_2(X) = kappa
                            (Section 5.1.1, the SVD-based matrix).
  * ``stacked_lower``    -- 400 stacked copies of a 50x50 lower-triangular F
                            with F_ii = 100, F_ij = a (j < i)
                            (Section 5.1.2).
  * ``arrowhead``        -- X = -5 e_b e_a^T + [diag(1,..,1,beta); 0]
                            (Section 5.1.3).
  * ``known_answer``     -- X = Q0 R0 with a chosen upper-triangular R0 of
                            positive diagonal, so the QR factors are known.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng",
    "orthonormal",
    "svd_matrix",
    "stacked_lower",
    "arrowhead",
    "known_answer",
    "integer_matrix",
    "gaussian_sketch",
    "sparse_sign_sketch",
    "kappa_seed",
    "batched_problems",
]


def rng(seed: int) -> np.random.Generator:
    """numpy Generator on the Philox bit generator, keyed by ``seed``."""
    return np.random.Generator(np.random.Philox(int(seed)))


def kappa_seed(config_index: int, kappa_index: int) -> int:
    """Seed convention for the benchmark matrices: 20241206 + 1000*config + kappa index."""
    return 20241206 + 1000 * int(config_index) + int(kappa_index)


def orthonormal(m: int, n: int, seed: int) -> np.ndarray:
    """Thin Q (m x n, orthonormal columns) from Householder QR of a seeded N(0,1) matrix."""
    g = rng(seed).standard_normal((m, n))
    q, r = np.linalg.qr(g, mode="reduced")
    # make the basis independent of LAPACK's sign convention
    q *= np.sign(np.diag(r))[None, :]
    return np.asfortranarray(q)


def svd_matrix(m: int, n: int, kappa: float, seed: int) -> np.ndarray:
    """X = U diag(sigma) V^T, sigma_i = kappa^(-(i)/(n-1)), i = 0..n-1.

    U: thin Q of a seeded N(0,1) m x n matrix; V: Q of a seeded N(0,1) n x n
    matrix (seed + 1).  ||X||_2 = 1 and kappa_2(X) = kappa up to rounding.
    """
    u = orthonormal(m, n, seed)
    v = orthonormal(n, n, seed + 1)
    if n > 1:
        sigma = np.power(float(kappa), -np.arange(n, dtype=np.float64) / (n - 1))
    else:
        sigma = np.ones(1)
    x = (u * sigma[None, :]) @ v.T
    return np.asfortranarray(x)


def stacked_lower(a: float, copies: int = 400, nb: int = 50) -> np.ndarray:
    """Stack ``copies`` copies of F (nb x nb): F_ii = 100, F_ij = a for j < i, else 0."""
    f = np.tril(np.full((nb, nb), float(a)), -1) + 100.0 * np.eye(nb)
    return np.asfortranarray(np.vstack([f] * copies))


def arrowhead(beta: float, m: int = 20000, n: int = 50) -> np.ndarray:
    """X = -5 e_b e_a^T + P_s with e_a = (0,1,...,1), e_b = e_1 and P_s = [diag(1,..,1,beta); 0]."""
    x = np.zeros((m, n))
    x[:n, :n] = np.diag(np.r_[np.ones(n - 1), float(beta)])
    x[0, 1:] += -5.0
    return np.asfortranarray(x)


def known_answer(m: int, n: int, seed: int, kappa_r: float = 1e3):
    """(X, Q0, R0) with X = Q0 R0 in exact arithmetic.

    Q0 has orthonormal columns; R0 = diag(d) (I + T) is upper triangular with
    a positive diagonal d geometric from 1 to 1/kappa_r and T strictly upper
    with N(0, 0.09/n) entries.
    The positive-diagonal thin QR is unique, so R must equal R0 and Q must
    equal Q0 up to the conditioning of the problem.
    """
    q0 = orthonormal(m, n, seed)
    g = rng(seed + 2)
    # R0 = diag(d) (I + T) with T strictly upper, N(0, 0.3^2/n) entries: the
    # unit factor stays well conditioned, so kappa(R0) stays near kappa_r.
    t = np.triu(g.standard_normal((n, n)), 1) * (0.3 / math.sqrt(max(n, 1)))
    if n > 1:
        d = np.power(float(kappa_r), -np.arange(n) / (n - 1))
    else:
        d = np.ones(1)
    r0 = d[:, None] * (np.eye(n) + t)
    x = np.asfortranarray(q0 @ r0)
    return x, q0, np.asfortranarray(r0)


def integer_matrix(m: int, n: int, seed: int, lo: int = -9, hi: int = 9) -> np.ndarray:
    """Small-integer matrix (exactly representable; used by brute-force pins)."""
    return np.asfortranarray(rng(seed).integers(lo, hi + 1, size=(m, n)).astype(np.float64))


def gaussian_sketch(s: int, m: int, seed: int) -> np.ndarray:
    """Explicit Gaussian sketch S (s x m, column-major) with N(0, 1/s) entries."""
    g = rng(seed).standard_normal((s, m))
    return np.asfortranarray(g / math.sqrt(s))


def sparse_sign_sketch(s: int, m: int, zeta: int, seed: int) -> np.ndarray:
    """Explicit sparse-sign sketch S (s x m, dense storage): each column has
    ``zeta`` distinct rows chosen uniformly, each +-1/sqrt(zeta) with a fair sign."""
    if zeta > s:
        raise ValueError("zeta must not exceed s")
    g = rng(seed)
    out = np.zeros((s, m))
    val = 1.0 / math.sqrt(zeta)
    for i in range(m):
        rows = g.choice(s, size=zeta, replace=False)
        signs = g.integers(0, 2, size=zeta) * 2 - 1
        out[rows, i] = signs * val
    return np.asfortranarray(out)


def batched_problems(count: int = 512, seed: int = None):
    """Sizes of the uneven batch of independent problems: m = floor(2^U(12,17)),
    n uniform in {16, 32, 48, 64, 96, 128}, kappa = 10^U(2,12) (the sketch size
    is s = 2n).  Returns (ms, ns, kappas) as numpy arrays; problem i's matrix
    is ``svd_matrix(ms[i], ns[i], kappas[i], seed + 1 + i)``."""
    if seed is None:
        seed = kappa_seed(3, 0)
    g = rng(seed)
    ms = np.floor(2.0 ** g.uniform(12, 17, count)).astype(np.int64)
    ns = g.choice(np.array([16, 32, 48, 64, 96, 128]), count)
    kap = 10.0 ** g.uniform(2, 12, count)
    return ms, ns, kap
