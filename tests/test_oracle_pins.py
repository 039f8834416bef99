"""Pins for the CPU oracle: each routine is checked against something other
than itself -- exact integer arithmetic, LAPACK (numpy/scipy), brute force in
50-digit arithmetic (mpmath), closed forms, published test vectors and the
paper's error bounds.  A dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of these.  No GPU is used."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _int_upper(n, seed, diag=(1, 3)):
    g = np.random.default_rng(seed)
    r = np.triu(g.integers(-4, 5, size=(n, n)), 1).astype(np.float64)
    r += np.diag(g.integers(diag[0], diag[1] + 1, size=n).astype(np.float64))
    return np.asfortranarray(r)


# ------------------------------------------------------------ Gram, TRMM ---

@pytest.mark.parametrize("m,n", [(1, 1), (7, 3), (130, 17), (257, 40)])
def test_gram_exact_on_integers(m, n):
    x = synth.integer_matrix(m, n, seed=m * 31 + n)
    xi = x.astype(np.int64)
    assert np.array_equal(oracle.gram(x), (xi.T @ xi).astype(np.float64))


def test_gram_is_xtx_not_xxt():
    x = synth.integer_matrix(9, 4, seed=3)
    g = oracle.gram(x)
    assert g.shape == (4, 4)
    assert np.array_equal(g, g.T)


@pytest.mark.parametrize("n", [1, 2, 5, 16])
def test_trmm_upper_exact(n):
    a = _int_upper(n, 1)
    b = _int_upper(n, 2)
    ref = (np.triu(a).astype(np.int64) @ np.triu(b).astype(np.int64)).astype(np.float64)
    assert np.array_equal(oracle.trmm_upper(a, b), ref)


# -------------------------------------------------------------- Cholesky ---

@pytest.mark.parametrize("n", [1, 3, 8, 24])
def test_cholesky_recovers_integer_factor_exactly(n):
    # G = R^T R with an integer R of positive diagonal: every quantity of the
    # column Cholesky is an exact integer, so R comes back bit for bit.
    r = _int_upper(n, 10 + n, diag=(1, 4))
    g = (r.T.astype(np.int64) @ r.astype(np.int64)).astype(np.float64)
    rr, st, _ = oracle.cholesky(g)
    assert st == 0
    assert np.array_equal(rr, r)


def test_cholesky_brute_force_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    g0 = np.random.default_rng(5).standard_normal((6, 6))
    g = g0.T @ g0 + 0.1 * np.eye(6)
    r, st, _ = oracle.cholesky(g)
    assert st == 0
    ref = mpmath.cholesky(mpmath.matrix(g.tolist()))  # lower L with G = L L^T
    ref_r = np.array([[float(ref[j, i]) for j in range(6)] for i in range(6)])
    assert np.max(np.abs(r - ref_r)) <= 1e-13 * np.max(np.abs(ref_r))


def test_cholesky_breakdown_status_and_column():
    g = np.diag([4.0, 1.0, -1.0, 2.0])
    _, st, info = oracle.cholesky(g, raise_on_error=False)
    assert st == oracle.CHOL_BREAKDOWN and info == 2
    g = np.array([[1.0, 2.0], [2.0, 1.0]])  # indefinite: radicand 1 - 4 < 0 at column 1
    _, st, info = oracle.cholesky(g, raise_on_error=False)
    assert st == oracle.CHOL_BREAKDOWN and info == 1
    g = np.array([[np.nan]])
    _, st, info = oracle.cholesky(g, raise_on_error=False)
    assert st == oracle.CHOL_BREAKDOWN and info == 0


# ------------------------------------------------------------------ TRSM ---

@pytest.mark.parametrize("m,n", [(1, 1), (11, 4), (200, 33)])
def test_trsm_exact_on_unit_integer_factor(m, n):
    # R integer upper with diagonal +-1, Q integer: X = Q R exactly and the
    # substitution X R^{-1} reproduces Q exactly.
    g = np.random.default_rng(m + n)
    r = np.triu(g.integers(-3, 4, size=(n, n)), 1).astype(np.float64)
    r += np.diag(g.choice([-1.0, 1.0], size=n))
    q = g.integers(-5, 6, size=(m, n)).astype(np.float64)
    x = (q.astype(np.int64) @ r.astype(np.int64)).astype(np.float64)
    assert np.array_equal(oracle.trsm(x, r), q)


def test_trsm_matches_lapack_triangular_solve():
    g = np.random.default_rng(9)
    n, m = 12, 50
    r = np.triu(g.standard_normal((n, n))) + 4 * np.eye(n)
    x = g.standard_normal((m, n))
    ref = scipy.linalg.solve_triangular(r.T, x.T, lower=True).T  # X R^{-1}
    assert np.max(np.abs(oracle.trsm(x, r) - ref)) <= 1e-13 * np.max(np.abs(ref))


# ------------------------------------------------------------------ GEPP ---

def _rational_gepp(a):
    """Exact GEPP over the rationals (first-index tie-break)."""
    a = [[Fraction(int(v)) for v in row] for row in a]
    m, n = len(a), len(a[0])
    piv = []
    for k in range(min(m, n)):
        p = max(range(k, m), key=lambda i: (abs(a[i][k]), -i))
        piv.append(p)
        a[k], a[p] = a[p], a[k]
        for i in range(k + 1, m):
            a[i][k] = a[i][k] / a[k][k]
            for j in range(k + 1, n):
                a[i][j] -= a[i][k] * a[k][j]
    return a, piv


@pytest.mark.parametrize("m,n,seed", [(5, 5, 1), (9, 4, 2), (16, 8, 3), (8, 8, 4)])
def test_gepp_brute_force_rational(m, n, seed):
    x = synth.integer_matrix(m, n, seed, lo=-6, hi=6)
    x[:, 0] += 50.0 * np.eye(m, n)[:, 0]  # keep it nonsingular
    ex, piv = _rational_gepp(x)
    lu, ipiv, st, _ = oracle.gepp(x)
    assert st == 0
    assert list(ipiv) == piv
    ref = np.array([[float(v) for v in row] for row in ex])
    assert np.max(np.abs(lu - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_gepp_tie_break_smallest_index():
    x = np.array([[1.0, 2.0], [-3.0, 1.0], [3.0, 5.0], [2.0, 0.0]])
    lu, ipiv, st, _ = oracle.gepp(x)
    assert ipiv[0] == 1  # |-3| == |3|: the first one wins


def test_gepp_matches_lapack_getrf():
    # well conditioned, so that LAPACK's blocked summation order and ours
    # agree to a few ulps; the pivot sequence must be identical
    x = synth.svd_matrix(300, 20, 10.0, 11)
    lu, ipiv, st, _ = oracle.gepp(x)
    lu_ref, piv_ref = scipy.linalg.lu_factor(x)
    assert np.array_equal(ipiv, piv_ref[:20])
    assert np.max(np.abs(lu - lu_ref[:, :20])) <= 1e-13


def test_gepp_backward_error_eq_elu():
    # |P X - M N| <= 1.02 n u |M||N|  (eq. (elu))
    x = synth.svd_matrix(400, 24, 1e8, 12)
    lu, ipiv, st, _ = oracle.gepp(x)
    px = x.copy()
    for k, p in enumerate(ipiv):
        px[[k, p]] = px[[p, k]]
    mm, nn = oracle.unit_lower(lu), oracle.upper(lu)
    err = np.abs(px - mm @ nn)
    bound = 1.02 * 24 * U * (np.abs(mm) @ np.abs(nn))
    assert np.all(err <= bound + 1e-300)
    assert np.max(np.abs(mm)) <= 1.0


def test_gepp_zero_pivot_reported():
    x = np.array([[1.0, 2.0], [2.0, 4.0], [3.0, 6.0]])
    _, _, st, info = oracle.gepp(x, raise_on_error=False)
    assert st == oracle.LU_ZERO_PIVOT and info == 1


# ----------------------------------------------------------- Householder ---

@pytest.mark.parametrize("s,n", [(1, 1), (6, 3), (40, 17), (128, 64)])
def test_householder_r_matches_lapack_including_signs(s, n):
    a = np.random.default_rng(s * n).standard_normal((s, n))
    r = oracle.householder_r(a)
    r_ref = np.linalg.qr(a, mode="r")  # dgeqrf: beta = -sign(alpha) ||x||
    assert np.allclose(r, np.triu(r_ref[:n]), rtol=0, atol=1e-13 * np.max(np.abs(r_ref)))


def test_householder_r_invariant_rtr_equals_ata():
    a = synth.svd_matrix(64, 10, 1e5, 4)
    r = oracle.householder_r(a)
    assert np.allclose(r.T @ r, a.T @ a, atol=1e-14)
    assert np.array_equal(r, np.triu(r))


def test_householder_skips_zero_subcolumn():
    a = np.array([[-2.0, 1.0], [0.0, 3.0], [0.0, 4.0]])
    r = oracle.householder_r(a)
    assert r[0, 0] == -2.0 and r[0, 1] == 1.0       # H_0 = I
    assert abs(abs(r[1, 1]) - 5.0) < 1e-15           # ||(3, 4)|| = 5, beta = -5
    assert r[1, 1] < 0


# ---------------------------------------------------------------- Givens ---
# The alternative R-factor of Section 1 and the remark after Algorithm 5.

@pytest.mark.parametrize("s,n", [(2, 1), (6, 3), (40, 17), (128, 64), (300, 128)])
def test_givens_r_is_lapack_r_with_nonnegative_diagonal(s, n):
    # s > n: every column has a subcolumn to rotate, so the diagonal is positive
    a = np.random.default_rng(s + 7 * n).standard_normal((s, n))
    r = oracle.givens_r(a)
    r_ref = np.triu(np.linalg.qr(a, mode="r")[:n])
    r_ref = np.sign(np.diag(r_ref))[:, None] * r_ref   # the unique positive-diagonal R
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert np.max(np.abs(r - r_ref)) <= 1e-13 * np.max(np.abs(r_ref))


def test_givens_r_brute_force_mpmath():
    for seed, (s, n) in enumerate([(5, 3), (9, 8), (12, 6)]):
        a = np.random.default_rng(100 + seed).standard_normal((s, n))
        _, r_mp = _mp_qr(a)
        r = oracle.givens_r(a)
        assert np.max(np.abs(r - r_mp)) <= 4e-15 * np.max(np.abs(r_mp)), (s, n)


def test_givens_r_closed_forms():
    # one column: r = ||a||; (3, 4) -> 5 exactly (hypot is exact there)
    assert oracle.givens_r(np.array([[3.0], [4.0]]))[0, 0] == 5.0
    a = np.random.default_rng(3).standard_normal((50, 1))
    assert abs(oracle.givens_r(a)[0, 0] - np.linalg.norm(a)) <= 4e-15 * np.linalg.norm(a)
    # an input that is already upper triangular needs no rotation: R = its top block
    u = np.triu(np.random.default_rng(4).standard_normal((6, 4)))
    u[:4][np.diag_indices(4)] = np.abs(np.diag(u[:4])) + 1.0
    assert np.array_equal(oracle.givens_r(u), u[:4])
    # a zero subcolumn keeps its diagonal sign (no rotation), like Householder's H_k = I
    a = np.array([[-2.0, 1.0], [0.0, 3.0], [0.0, 4.0]])
    r = oracle.givens_r(a)
    assert r[0, 0] == -2.0 and r[0, 1] == 1.0 and r[1, 1] == 5.0


def test_givens_r_invariant_and_householder_agreement():
    a = synth.svd_matrix(64, 10, 1e5, 4)
    rg, rh = oracle.givens_r(a), oracle.householder_r(a)
    assert np.allclose(rg.T @ rg, a.T @ a, atol=1e-14)
    d = np.sign(np.diag(rh))[:, None]
    assert np.max(np.abs(rg - d * rh)) <= 1e-13 * np.max(np.abs(rh))


@pytest.mark.parametrize("name", ["rclupp", "rcluppr", "rcholqr"])
def test_drivers_with_givens_r0_match_householder(name):
    m, n = 2000, 24
    x = synth.svd_matrix(m, n, 1e6, 8)
    S = synth.gaussian_sketch(2 * n, m, 9)
    fn = getattr(oracle, name)
    qg, rg, st = fn(x, S=S, r0="givens")
    qh, rh, _ = fn(x, S=S)
    assert st == 0
    assert oracle.orthogonality(qg) <= max(2 * oracle.orthogonality(qh), 1e-14)
    assert oracle.residual(x, qg, rg) <= max(2 * oracle.residual(x, qh, rh), 1e-15)
    assert np.linalg.norm(rg - rh) / np.linalg.norm(rh) <= 1e-10 * 1e6
    r1g, _, _ = oracle.sketch_precond(oracle.sketch_dense(S, x), r0="givens")
    r1h, _, _ = oracle.sketch_precond(oracle.sketch_dense(S, x))
    assert np.max(np.abs(r1g - r1h)) <= 1e-12 * np.max(np.abs(r1h))


# --------------------------------------------------------------- sketches ---

def test_sketch_dense_exact_on_integers():
    g = np.random.default_rng(3)
    S = g.integers(-3, 4, size=(7, 50)).astype(np.float64)
    x = g.integers(-5, 6, size=(50, 6)).astype(np.float64)
    ref = (S.astype(np.int64) @ x.astype(np.int64)).astype(np.float64)
    assert np.array_equal(oracle.sketch_dense(S, x), ref)


def test_sketch_sparse_equals_dense_definition():
    s, m, zeta = 16, 300, 4  # 1/sqrt(4) = 1/2: exact
    rows, signs = oracle.sparse_sign_pattern(s, m, zeta, seed=77)
    x = synth.integer_matrix(m, 5, 8)
    S = oracle.sparse_to_dense(s, m, zeta, rows, signs)
    y1 = oracle.sketch_sparse(s, zeta, rows, signs, x)
    y2 = oracle.sketch_dense(S, x)
    ref = (2 * S).astype(np.int64) @ x.astype(np.int64) / 2.0
    assert np.array_equal(y1, ref) and np.array_equal(y2, ref)


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t, 16) for t in line.split()]
                rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(oracle.philox4x32_10(ctr, key)) == out


def test_ln_and_cossin_definitions_are_accurate():
    xs = np.concatenate([np.arange(1, 2 ** 23, 9973) * 2.0 ** -23, [2.0 ** -23, 0.5, 1.0]])
    for x in xs.astype(np.float32):
        assert abs(oracle.ln_f32(float(x)) - math.log(float(x))) <= 4e-7 * max(1.0, abs(math.log(float(x))))
    for u in np.arange(0, 2 ** 23, 7919) * 2.0 ** -23:
        c, s = oracle.cossin_2pi_f32(float(np.float32(u)))
        assert abs(c - math.cos(2 * math.pi * u)) < 1e-6
        assert abs(s - math.sin(2 * math.pi * u)) < 1e-6
    assert oracle.ln_f32(1.0) == 0.0
    assert oracle.cossin_2pi_f32(0.0) == (1.0, 0.0)


def test_gaussian_sketch_statistics():
    from scipy import stats
    z = np.array([oracle.gauss_entry(123, r, i) for r in range(8) for i in range(4000)])
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1.0) < 0.04
    assert stats.kstest(z, "norm").pvalue > 1e-3
    S = oracle.gaussian_sketch_matrix(32, 1000, 5)
    assert abs(np.mean(np.sum(S * S, axis=0)) - 1.0) < 0.05  # column norms ~ 1 (N(0, 1/s))
    # the same (seed, r, i) always gives the same entry
    assert oracle.gauss_entry(123, 5, 17) == oracle.gauss_entry(123, 5, 17)
    assert oracle.gauss_entry(123, 5, 17) != oracle.gauss_entry(124, 5, 17)


def test_gaussian_sketch_rows_are_uncorrelated():
    # S = G / sqrt(s) with G's entries independent (Section 3): across many
    # columns, the sample correlation of any two rows is O(1/sqrt(columns)).
    # Rows 4b .. 4b+3 share one Philox block, so this also pins that each
    # lane draws its own value from the block.
    cols = 20000
    S = oracle.gaussian_sketch_matrix(8, cols, 31)
    c = np.corrcoef(S)
    off = c[~np.eye(8, dtype=bool)]
    assert np.max(np.abs(off)) < 6.0 / math.sqrt(cols)


def test_cholqr2_stage_recovers_from_a_weak_sketch():
    # A sketch that only sees the first s rows, where X's first column is 1e-4
    # times smaller than elsewhere, is a poor embedding for this X: Q1 = X R1^-1
    # has kappa ~ 6e4 (a Gaussian s = 2n sketch gives ~ 5), and not by a column
    # scaling -- the under-sketched direction lies along the first row of
    # R1^-1, which mixes all columns -- so the first CholeskyQR pass leaves
    # Q2 visibly non-orthogonal and R4 far from I.  CholeskyQR2 still returns
    # an orthonormal Q while kappa(Q1) is far below u^(-1/2) (Lemma 3.1), and R
    # = R4 R2 R1 (C4, C8) is X's R-factor to first order in kappa(Q1) u.
    m, n, s = 3000, 16, 32
    u = 2.0 ** -53
    rng = np.random.default_rng(91)
    x = rng.standard_normal((m, n))
    x[:s, 0] *= 1e-4
    S = np.zeros((s, m))
    S[:, :s] = rng.standard_normal((s, s)) / math.sqrt(s)
    R1, _, _ = oracle.sketch_precond(S @ x)
    Q1 = oracle.trsm(x, R1)
    k1 = np.linalg.cond(Q1 / np.sqrt(np.sum(Q1 * Q1, axis=0)))  # after column equilibration
    assert k1 > 1e4
    rh = np.linalg.qr(x, mode="r")
    rh = np.sign(np.diag(rh))[:, None] * rh
    q, r, _ = oracle.rclupp(x, S=S)
    assert oracle.orthogonality(q) <= 1e-13
    assert oracle.residual(x, q, r) <= 20 * k1 * u
    assert np.linalg.norm(r - rh) <= 20 * k1 * u * np.linalg.norm(rh)


@pytest.mark.parametrize("kappa", [1e4, 1e12])
def test_rcluppr_preconditioner_is_the_r_factor_of_the_sketched_pivoted_x(kappa):
    # Algorithm 7: [M, N, P] = LU(X), R1 = R(S M) N.  P X = M N and N is upper
    # triangular, so R(S M) N = R(S M N) = R(S P X) up to row signs: the
    # preconditioner of Algorithm 6 for the row-permuted X.  Q1 = X R1^-1 is
    # then as well conditioned as a Gaussian sketch with s = 2n makes it
    # (about (1 + sqrt(n/s)) / (1 - sqrt(n/s)) ~ 5.8), whatever kappa(X) is.
    from scipy import linalg as sla
    m, n = 2000, 32
    x = synth.svd_matrix(m, n, kappa, 5)
    S = oracle.gaussian_sketch_matrix(2 * n, m, 3)
    R1, _, _ = oracle.rcluppr_precond(x, S=S)
    assert np.array_equal(R1, np.triu(R1)) and np.all(np.diag(R1) > 0)
    assert np.linalg.cond(np.linalg.solve(R1.T, x.T).T) <= 20
    P, _, _ = sla.lu(x)  # x = P L U: LAPACK getrf's pivots, which GEPP reproduces
    ref = np.linalg.qr(S @ (P.T @ x), mode="r")
    ref = np.sign(np.diag(ref))[:, None] * ref
    assert np.linalg.norm(R1 - ref) <= 1e-12 * np.linalg.norm(ref)


def test_sparse_signs_are_independent_of_the_rows():
    # The sparse-sign sketch draws each nonzero's row and its sign
    # independently (a fair sign, Section 3's CountSketch with zeta = 1): for
    # every row, the signs that land in it average to ~0.
    s, m, zeta = 64, 20000, 8
    rows, signs = oracle.sparse_sign_pattern(s, m, zeta, seed=5)
    rows, signs = np.asarray(rows).ravel(), np.asarray(signs).ravel().astype(np.float64)
    for r in range(s):
        sel = signs[rows == r]
        assert len(sel) > 1000 and abs(sel.mean()) < 5.0 / math.sqrt(len(sel)), r


def test_sparse_sign_pattern_properties():
    s, m, zeta = 64, 5000, 8
    rows, signs = oracle.sparse_sign_pattern(s, m, zeta, seed=3)
    r = rows.reshape(m, zeta)
    assert all(len(set(rr)) == zeta for rr in r)
    assert set(np.unique(signs)) == {-1, 1}
    counts = np.bincount(rows, minlength=s)
    from scipy import stats
    assert stats.chisquare(counts).pvalue > 1e-3
    S = oracle.sparse_to_dense(s, m, zeta, rows, signs)
    assert np.allclose(np.sum(S * S, axis=0), 1.0)
    # zeta == s forces the fallback path; it must still give distinct rows
    rows2, _ = oracle.sparse_sign_pattern(8, 20, 8, seed=1)
    assert all(sorted(rr) == list(range(8)) for rr in rows2.reshape(20, 8))


@pytest.mark.parametrize("kind", ["gauss", "sparse"])
def test_sketch_is_an_embedding_eq_s2(kind):
    # For X with orthonormal columns, the singular values of S X lie in
    # [sqrt(1-eps), sqrt(1+eps)] with eps = 0.5 (eq. (s2)), with high probability.
    # For a Gaussian S the extreme singular values sit near 1 +- sqrt(n/s), so
    # eps = 0.5 needs s >~ 20 n; s = 32 n here.
    m, n, s = 3000, 8, 256
    x = synth.orthonormal(m, n, 21)
    if kind == "gauss":
        y = oracle.sketch_dense(oracle.gaussian_sketch_matrix(s, m, 9), x)
    else:
        rows, signs = oracle.sparse_sign_pattern(s, m, 8, 9)
        y = oracle.sketch_sparse(s, 8, rows, signs, x)
    sv = np.linalg.svd(y, compute_uv=False)
    assert sv.max() <= math.sqrt(1.5) and sv.min() >= math.sqrt(0.5)


def test_sketch_precond_r1_is_r_factor_of_sketch():
    # R1 = R0 N is the R-factor of Y up to row signs; after the sign fix it is
    # the positive-diagonal one: R1^T R1 = Y^T Y and R1 = D R_householder(Y).
    y = synth.svd_matrix(64, 12, 1e4, 31)
    r1, st, _ = oracle.sketch_precond(y)
    rh = np.linalg.qr(y, mode="r")
    rh = np.sign(np.diag(rh))[:, None] * rh
    assert np.all(np.diag(r1) > 0) and np.array_equal(r1, np.triu(r1))
    assert np.max(np.abs(r1 - rh)) <= 1e-10 * np.max(np.abs(rh))


# ---------------------------------------------------------------- drivers ---

def _mp_qr(x):
    """Positive-diagonal thin QR in 50-digit arithmetic (Cholesky of the exact Gram)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    X = mpmath.matrix(x.tolist())
    G = X.T * X
    L = mpmath.cholesky(G)
    R = L.T
    Q = X * R ** -1
    m, n = x.shape
    return (np.array([[float(Q[i, j]) for j in range(n)] for i in range(m)]),
            np.array([[float(R[i, j]) for j in range(n)] for i in range(n)]))


def _drivers(s):
    return {
        "cholqr2": lambda x: oracle.cholqr2(x),
        "lc2": lambda x: oracle.lc2(x),
        "rclupp": lambda x: oracle.rclupp(x, S=synth.gaussian_sketch(s, x.shape[0], 4)),
        "rcluppr": lambda x: oracle.rcluppr(x, S=synth.gaussian_sketch(s, x.shape[0], 4)),
        "rclupp_sparse": lambda x: oracle.rclupp(x, sparse=(s, 4) + oracle.sparse_sign_pattern(s, x.shape[0], 4, 4)),
        "rcluppr_sparse": lambda x: oracle.rcluppr(x, sparse=(s, 4) + oracle.sparse_sign_pattern(s, x.shape[0], 4, 4)),
    }


@pytest.mark.parametrize("name", list(_drivers(16)))
@pytest.mark.parametrize("n", [1, 3, 8])
def test_drivers_brute_force_small(name, n):
    x = synth.svd_matrix(40, n, 1e3, 100 + n)
    q_ref, r_ref = _mp_qr(x)
    q, r, st = _drivers(max(2 * n, 4))[name](x)
    assert st == 0
    assert np.max(np.abs(r - r_ref)) <= 1e-12 * np.max(np.abs(r_ref))
    assert np.max(np.abs(q - q_ref)) <= 1e-11


@pytest.mark.parametrize("name", list(_drivers(64)))
def test_drivers_known_answer(name):
    x, q0, r0 = synth.known_answer(2000, 24, seed=8, kappa_r=1e4)
    q, r, st = _drivers(64)[name](x)
    assert st == 0
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert np.linalg.norm(r - r0) / np.linalg.norm(r0) <= 1e-12 * 1e4
    assert np.max(np.abs(q - q0)) <= 1e-10


@pytest.mark.parametrize("name", list(_drivers(100)))
def test_drivers_agree_with_householder_up_to_signs(name):
    x = synth.svd_matrix(2000, 50, 1e6, 13)
    q, r, st = _drivers(100)[name](x)
    qh, rh = np.linalg.qr(x)
    d = np.sign(np.diag(rh))
    rh, qh = d[:, None] * rh, qh * d[None, :]
    assert np.linalg.norm(r - rh) / np.linalg.norm(rh) <= 1e-15 * 1e6 * 10
    assert np.linalg.norm(q - qh) <= 1e-15 * 1e6 * 10


@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10])
def test_singular_values_of_r_closed_form(kappa):
    # X = U diag(sigma) V^T: R has the singular values sigma (R^T R = V S^2 V^T).
    m, n = 3000, 20
    x = synth.svd_matrix(m, n, kappa, 41)
    q, r, st = oracle.rclupp(x, S=synth.gaussian_sketch(40, m, 2))
    sv = np.linalg.svd(r, compute_uv=False)
    sigma = np.power(kappa, -np.arange(n) / (n - 1))
    assert np.max(np.abs(sv - sigma) / sigma) <= 1e-15 * kappa * 100


def _thm41_bounds(m, n, x, eps=0.5):
    h = 1.0 / (0.78 / math.sqrt(1 + eps) - 0.1 / math.sqrt(1 - eps))
    orth = 6 * (m * n * U + n * (n + 1) * U)
    res = (4.36 / math.sqrt(1 - eps) * h * n * math.sqrt(n) * U * np.linalg.norm(x, "fro")
           + 3.02 / math.sqrt(1 - eps) * h * n * n * U * np.linalg.norm(x, 2))
    return orth, res


@pytest.mark.parametrize("kappa", [1e4, 1e8, 1e12])
@pytest.mark.parametrize("algo", ["rclupp", "rcluppr"])
def test_theorem_4_1_bounds(kappa, algo):
    m, n, s = 4096, 64, 128
    x = synth.svd_matrix(m, n, kappa, 51)
    S = synth.gaussian_sketch(s, m, 52)
    q, r, st = getattr(oracle, algo)(x, S=S)
    orth_b, res_b = _thm41_bounds(m, n, x)
    assert oracle.orthogonality(q) <= orth_b
    assert np.linalg.norm(q @ r - x, "fro") <= res_b


def test_cholqr2_lemma_3_1_and_breakdown():
    m, n = 4096, 32
    x = synth.svd_matrix(m, n, 1e3, 61)
    q, r, st = oracle.cholqr2(x)
    assert oracle.orthogonality(q) <= 6 * (m * n * U + n * (n + 1) * U)
    assert np.linalg.norm(q @ r - x, "fro") <= 5 * n ** 2.5 * U * np.linalg.norm(x, 2)
    # kappa beyond u^{-1/2}: CholeskyQR2 breaks down (Section 2.2)
    _, _, st = oracle.cholqr2(synth.svd_matrix(m, n, 1e12, 62), raise_on_error=False)
    assert st == oracle.CHOL_BREAKDOWN


def test_lc2_lemma_3_3():
    m, n = 4096, 32
    x = synth.svd_matrix(m, n, 1e6, 71)
    q, r, st = oracle.lc2(x)
    assert oracle.orthogonality(q) <= 6.5 * (m * n * U + n * (n + 1) * U)
    assert np.linalg.norm(q @ r - x, "fro") <= 4.09 * n * n * U * np.linalg.norm(x, 2)


def test_rcluppr_robust_on_arrowhead_section_5_1_3():
    # The arrowhead matrix of Section 5.1.3: RCLUPPr stays accurate where
    # CholeskyQR2 breaks down.
    x = synth.arrowhead(1e-10, m=2000, n=20)
    q, r, st = oracle.rcluppr(x, S=synth.gaussian_sketch(40, 2000, 3))
    assert st == 0 and oracle.orthogonality(q) < 1e-12 and oracle.residual(x, q, r) < 1e-14
    _, _, st2 = oracle.cholqr2(x, raise_on_error=False)
    assert st2 == oracle.CHOL_BREAKDOWN


def test_stacked_lower_section_5_1_2():
    x = synth.stacked_lower(-0.8, copies=40, nb=20)
    for algo in ("rclupp", "rcluppr"):
        q, r, st = getattr(oracle, algo)(x, S=synth.gaussian_sketch(40, x.shape[0], 3))
        assert st == 0 and oracle.orthogonality(q) < 1e-12 and oracle.residual(x, q, r) < 1e-14


# ------------------------------------------- reduced-precision sketch tier ---

def _rne_bf16_reference(x):
    # independent formula: x = f 2^e, f in [0.5, 1); keep 8 bits of f with
    # Python's round() (ties to even on exactly representable halves)
    if x == 0.0:
        return 0.0
    f, e = math.frexp(x)
    return math.ldexp(round(f * 256.0), e - 8)


def test_round_bf16_against_independent_formula():
    g = np.random.default_rng(17)
    vals = np.concatenate([g.standard_normal(2000) * 10.0 ** g.integers(-30, 30, 2000),
                           [1.0, -1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, 255.5, 256.5, 1e-30]])
    for v in vals:
        assert oracle.round_bf16(float(v)) == _rne_bf16_reference(float(v)), v
    # ties: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even (1.0)
    assert oracle.round_bf16(1.0 + 2 ** -8) == 1.0
    assert oracle.round_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6


def test_bf16_split_keeps_24_bits():
    x = synth.rng(3).standard_normal(5000)
    xs = oracle.bf16_split(x, 3)
    assert np.all(np.abs(x - xs) <= 2.0 ** -23 * np.abs(x))
    x1 = oracle.bf16_split(x, 1)
    assert np.all(np.abs(x - x1) <= 2.0 ** -8 * np.abs(x))


def test_tier_levels_against_library_quantile():
    # T[j] = round(32 Phi^{-1}((j + 1/2) / 4096)) / 32: scipy's ndtri (an
    # independent implementation of the normal quantile) gives every level,
    # numpy's rint (half to even) the rounding
    from scipy.special import ndtri
    t = oracle.tier_levels()
    ref = np.rint(32.0 * ndtri((np.arange(4096) + 0.5) / 4096)) / 32.0
    assert np.array_equal(t, ref)
    # symmetric, increasing, integers over 32 within bf16's 8 bits, zero as +0,
    # and a unit variance up to the discretisation
    assert np.array_equal(t, -t[::-1] + 0.0) and np.all(np.diff(t) >= 0)
    k = 32 * t
    assert np.array_equal(k, np.round(k)) and np.max(np.abs(k)) <= 128
    assert not np.any(np.signbit(t[t == 0]))
    assert abs(t.var() - 1.0) < 2e-3
    # the quantile itself at closed-form points
    assert oracle.normal_quantile(0.5 - 1e-17) <= 0.0
    assert abs(oracle.normal_quantile(0.8413447460685429) - 1.0) < 1e-12
    assert abs(oracle.normal_quantile(0.022750131948179195) + 2.0) < 1e-12


def test_tier_sketch_entries_follow_philox():
    # entry (r, i) = T[top 12 bits of 16-bit half (i mod 8) mod 2 of word
    # (i mod 8) div 2 of Philox4x32-10 at counter (i div 8, 0, r, 0x53424631)]
    # -- Philox itself is pinned by its known-answer vectors
    t = oracle.tier_levels()
    seed, s, m = 0x1234_5678_9ABC, 5, 37
    z = oracle.tier_sketch_z(s, m, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for r in range(s):
        for i in range(m):
            w = oracle.philox4x32_10([i // 8, 0, r, 0x53424631], key)
            h = (int(w[(i % 8) // 2]) >> (16 * (i % 2))) & 0xFFFF
            assert z[r, i] == t[h >> 4], (r, i)


def test_tier_sketch_statistics():
    # uniform table indices, independent entries across rows and along a row
    # (the eight entries of one Philox block are separate draws), unit variance
    from scipy import stats
    z = oracle.tier_sketch_z(16, 20000, 77)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    t = oracle.tier_levels()
    lv = np.unique(t)
    counts = np.bincount(np.searchsorted(lv, z.ravel()), minlength=len(lv))
    expect = np.array([np.sum(t == v) for v in lv], dtype=np.float64) / 4096 * z.size
    assert stats.chisquare(counts, expect).pvalue > 1e-4
    c = np.corrcoef(z)
    assert np.max(np.abs(c[~np.eye(16, dtype=bool)])) < 6.0 / math.sqrt(20000)
    lag = [np.corrcoef(z[:, :-d].ravel(), z[:, d:].ravel())[0, 1] for d in range(1, 9)]
    assert np.max(np.abs(lag)) < 6.0 / math.sqrt(z.size)


@pytest.mark.parametrize("nterms", [1, 3])
def test_sketch_bf16_definition(nterms):
    m, n, s, seed = 700, 9, 24, 5
    x = synth.svd_matrix(m, n, 1e3, 2)
    y = oracle.sketch_bf16(s, seed, nterms, x)
    z = oracle.tier_sketch_z(s, m, seed)
    ref = oracle.sketch_dense(z, oracle.bf16_split(x, nterms)) / math.sqrt(s)
    assert np.allclose(y, ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))
    # exact on integers: small-integer X is its own bf16 split, and every
    # product and sum of bf16 levels times small integers is exact in binary64
    xi = synth.integer_matrix(300, 4, 8)
    yi = oracle.sketch_bf16(s, seed, nterms, xi)
    zi = oracle.tier_sketch_z(s, 300, seed)
    assert np.array_equal(yi, (zi @ xi) * (1.0 / math.sqrt(s)))


def test_tier_sketch_is_an_embedding_eq_s2():
    # the discretised normal is sub-Gaussian with (nearly) unit variance, so
    # z_b / sqrt(s) embeds like the Gaussian sketch (eq. (s2), eps = 0.5)
    m, n, s = 3000, 8, 256
    x = synth.orthonormal(m, n, 21)
    y = oracle.sketch_dense(oracle.tier_sketch_z(s, m, 9) / math.sqrt(s), x)
    sv = np.linalg.svd(y, compute_uv=False)
    assert sv.max() <= math.sqrt(1.5) and sv.min() >= math.sqrt(0.5)


def test_sketch_digits_exact_on_integers():
    # small integers are their own six-digit rounding, and k x sums exactly:
    # Y = (k X) 2^-5 / sqrt(s) with one rounding of the exact sum
    s, seed = 24, 7
    x = synth.integer_matrix(500, 6, 3)
    y = oracle.sketch_digits(s, seed, x)
    k = 32 * oracle.tier_sketch_z(s, 500, seed)
    assert np.array_equal(y, ((k @ x) * 2.0 ** -5) * (1.0 / math.sqrt(s)))


def test_sketch_digits_rounds_x_to_48_bits_of_its_column():
    # a column with largest entry in [1, 2) has E = 1 and keeps 2^-46 steps,
    # rounding half away from zero: 1 + 2^-47 -> 1 + 2^-46, 1 + 2^-48 -> 1
    s, seed = 8, 11
    k = 32 * oracle.tier_sketch_z(s, 4, seed)
    cols = {1.0 + 2.0 ** -47: 1.0 + 2.0 ** -46, 1.0 + 2.0 ** -48: 1.0,
            -(1.0 + 2.0 ** -47): -(1.0 + 2.0 ** -46), 1.5 + 3 * 2.0 ** -48: 1.5 + 2.0 ** -46}
    for v, kept in cols.items():
        x = np.array([[v], [1.25], [-1.0], [0.5]])
        F = [int(f) for f in np.array([kept, 1.25, -1.0, 0.5]) * 2.0 ** 46]  # exact integers
        y = oracle.sketch_digits(s, seed, x)
        # the exact integer sum (Python integers), rounded once to binary64
        ref = [math.ldexp(float(sum(int(k[r, i]) * F[i] for i in range(4))), -51) * (1.0 / math.sqrt(s))
               for r in range(s)]
        assert np.array_equal(y[:, 0], np.array(ref)), v
    # a NaN makes its column NaN, the others stay finite
    x = np.ones((4, 2))
    x[2, 1] = np.nan
    y = oracle.sketch_digits(s, seed, x)
    assert np.all(np.isfinite(y[:, 0])) and np.all(np.isnan(y[:, 1]))


def test_sketch_digits_close_to_the_binary64_product():
    # |Y - z_b X / sqrt(s)| <= (2^-48 max_i |x_ij| sum_i |k_ri| / 32 + binary64
    # rounding of the reference) / sqrt(s): 48 bits of each column kept
    m, n, s, seed = 2000, 7, 32, 4
    x = synth.svd_matrix(m, n, 1e6, 9) * np.array([1e-200, 1.0, 3.0, 1e100, 1e-3, 7.0, 1e5])
    y = oracle.sketch_digits(s, seed, x)
    z = oracle.tier_sketch_z(s, m, seed)
    ref = oracle.sketch_dense(z, x) / math.sqrt(s)
    cmax = np.max(np.abs(x), axis=0)
    bound = (2.0 ** -48 * np.abs(z).sum(axis=1)[:, None] * cmax[None, :]
             + 4 * m * 2.0 ** -53 * (np.abs(z) @ np.abs(x))) / math.sqrt(s)
    assert np.all(np.abs(y - ref) <= bound)
    # and scaling a column by a power of two scales its sketch exactly
    x2 = x * np.array([2.0 ** 300, 1, 1, 2.0 ** -500, 1, 1, 1])
    y2 = oracle.sketch_digits(s, seed, x2)
    assert np.array_equal(y2, y * np.array([2.0 ** 300, 1, 1, 2.0 ** -500, 1, 1, 1]))


# ------------------------------------- comparison paths (Algorithms 3, 5) ---

def test_scholqr3_shift_closed_form():
    m, n = 1000, 7
    x = synth.integer_matrix(m, n, 4)
    g = oracle.gram(x)
    s = oracle.scholqr3_shift(m, g)
    col_norm2 = np.max(np.sum(x * x, axis=0))       # ||X||_g^2 (Definition 2.1)
    assert s == 11.0 * (m * n * U + n * (n + 1) * U) * col_norm2


@pytest.mark.parametrize("name", ["rcholqr", "scholqr3"])
@pytest.mark.parametrize("n", [1, 3, 8])
def test_comparison_paths_brute_force(name, n):
    x = synth.svd_matrix(40, n, 1e3, 200 + n)
    q_ref, r_ref = _mp_qr(x)
    if name == "rcholqr":
        q, r, st = oracle.rcholqr(x, S=synth.gaussian_sketch(max(2 * n, 4), 40, 4))
    else:
        q, r, st = oracle.scholqr3(x)
    assert np.max(np.abs(r - r_ref)) <= 1e-12 * np.max(np.abs(r_ref))
    assert np.max(np.abs(q - q_ref)) <= 1e-11


def test_scholqr3_lemma_3_2():
    # orthogonality 6(mnu + n(n+1)u) and residual 6.57 n^2 u ||X||_g + 4.81 n^2 u ||X||_2
    m, n = 4096, 32
    x = synth.svd_matrix(m, n, 1e6, 81)
    q, r, st = oracle.scholqr3(x)
    assert oracle.orthogonality(q) <= 6 * (m * n * U + n * (n + 1) * U)
    xg = np.max(np.linalg.norm(x, axis=0))
    assert np.linalg.norm(q @ r - x, "fro") <= 6.57 * n * n * U * xg + 4.81 * n * n * U * 1.0


def test_rcholqr_orthogonality_worse_than_rclupp_when_ill_conditioned():
    # Section 5.1: RCholeskyQR's single CholeskyQR leaves worse orthogonality
    # than RCLUPP on ill-conditioned X (qualitative claim)
    m, n = 4096, 32
    x = synth.svd_matrix(m, n, 1e12, 82)
    S = synth.gaussian_sketch(64, m, 83)
    q1, r1, st1 = oracle.rcholqr(x, S=S, raise_on_error=False)
    q2, r2, st2 = oracle.rclupp(x, S=S)
    assert st2 == 0
    if st1 == 0:
        assert oracle.orthogonality(q1) > oracle.orthogonality(q2)


def test_scholqr3_breaks_down_where_rclupp_does_not():
    # Section 2.2 / 5.1: SCholeskyQR3 fails as kappa approaches 1/u
    m, n = 2000, 20
    x = synth.svd_matrix(m, n, 1e15, 84)
    q, r, st = oracle.scholqr3(x, raise_on_error=False)
    ok = st == 0 and oracle.orthogonality(q) < 1e-10
    q2, r2, st2 = oracle.rcluppr(x, S=synth.gaussian_sketch(40, m, 85))
    assert st2 == 0 and oracle.orthogonality(q2) < 1e-12
    assert not ok or oracle.orthogonality(q) > oracle.orthogonality(q2)
