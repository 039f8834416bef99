"""Parity of the CUDA path (through the C ABI) with the CPU oracle, step by
step and algorithm by algorithm, on the same seeded inputs and the same
sketch.  Floating-point tolerances follow from the arithmetic:

  * a sum of m products computed in any order is within gamma_m (|a||b|)
    of the exact value (gamma_m = m u / (1 - m u)), so two such sums differ
    by at most 2 gamma_m (|a||b|) entrywise;
  * triangular solves / Cholesky differ by a forward error of order
    n u kappa (normwise);
  * whole factorizations are gated as the method's own accuracy requires:
    ||Q^T Q - I||_F and ||QR - X||_F / ||X||_F within max(10x oracle, 1e-13),
    and ||R - R_oracle||_F / ||R_oracle||_F <= 1e-10 kappa for kappa <= 1e6.

Integer and index results (pivot rows, exact-integer products) are bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def gamma(k):
    return k * U / (1 - k * U)


def dev(a):
    import paper_2412_06551_gb300 as rq
    a = np.asfortranarray(a, dtype=np.float64)
    t = torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda").t()
    assert t.stride(0) == 1
    return t


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


@pytest.fixture(scope="module")
def rq():
    import paper_2412_06551_gb300 as m
    m.load()
    return m


# ----------------------------------------------------------------- sketch ---

@pytest.mark.parametrize("m,n,s", [(1, 1, 1), (97, 5, 8), (1000, 17, 40), (4096, 64, 128),
                                   (10007, 128, 256), (3000, 200, 400)])
def test_sketch_explicit_S(rq, m, n, s):
    x = synth.svd_matrix(m, n, 1e3, m + n) if m >= n else synth.integer_matrix(m, n, 1)
    S = synth.gaussian_sketch(s, m, 5)
    y = host(rq.rclupp_sketch(dev(x), s=s, S=dev(S)))
    ref = oracle.sketch_dense(S, x)
    tol = 2 * gamma(m) * (np.abs(S) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - ref) <= tol)


@pytest.mark.parametrize("m,n,s,seed", [(5000, 32, 64, 0), (4096, 64, 128, 123), (777, 3, 17, 9),
                                        (20001, 128, 256, 2 ** 40 + 5)])
def test_sketch_gaussian_generator_matches_oracle(rq, m, n, s, seed):
    # The on-the-fly S equals the oracle's implementation of the same
    # counter-based definition bit for bit, so Y agrees to rounding.
    x = synth.svd_matrix(m, n, 1e2, 3)
    y = host(rq.rclupp_sketch(dev(x), s=s, seed=seed))
    S = oracle.gaussian_sketch_matrix(s, m, seed)
    ref = oracle.sketch_dense(S, x)
    tol = 2 * gamma(m) * (np.abs(S) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - ref) <= tol)


@pytest.mark.parametrize("m,n,s,zeta,seed", [(5000, 32, 64, 8, 0), (4099, 64, 256, 8, 11),
                                             (1000, 7, 16, 16, 3), (333, 40, 64, 1, 5)])
def test_sketch_sparse_sign_matches_oracle(rq, m, n, s, zeta, seed):
    x = synth.svd_matrix(m, n, 1e2, 4)
    y = host(rq.rclupp_sketch(dev(x), s=s, kind=rq.SKETCH_SPARSE_SIGN, zeta=zeta, seed=seed))
    rows, signs = oracle.sparse_sign_pattern(s, m, zeta, seed)
    ref = oracle.sketch_sparse(s, zeta, rows, signs, x)
    S = oracle.sparse_to_dense(s, m, zeta, rows, signs)
    tol = 2 * gamma(m) * (np.abs(S) @ np.abs(x)) + 1e-300
    assert np.all(np.abs(y - ref) <= tol)


@pytest.mark.parametrize("kind", [0, 1])
def test_sketch_of_unit_lower_factor(rq, kind):
    m, n, s = 3000, 24, 48
    x = synth.svd_matrix(m, n, 1e4, 8)
    lu, ipiv, st, _ = oracle.gepp(x)
    M = oracle.unit_lower(lu)
    y = host(rq.rclupp_sketch(dev(lu), s=s, kind=kind, seed=4, unit_lower=True))
    if kind == 0:
        S = oracle.gaussian_sketch_matrix(s, m, 4)
        ref = oracle.sketch_dense(S, M)
    else:
        rows, signs = oracle.sparse_sign_pattern(s, m, 8, 4)
        ref = oracle.sketch_sparse(s, 8, rows, signs, M)
        S = oracle.sparse_to_dense(s, m, 8, rows, signs)
    tol = 2 * gamma(m) * (np.abs(S) @ np.abs(M)) + 1e-300
    assert np.all(np.abs(y - ref) <= tol)


# ------------------------------------------------------------ Gram, TRSM ---

@pytest.mark.parametrize("m,n", [(1, 1), (63, 7), (1000, 16), (4097, 64), (5000, 100), (3001, 129),
                                 (2048, 256)])
def test_gram(rq, m, n):
    x = synth.svd_matrix(m, n, 1e4, 7) if m >= n else synth.integer_matrix(m, n, 2)
    g = host(rq.rclupp_gram(dev(x)))
    ref = oracle.gram(x)
    tol = 2 * gamma(m) * (np.abs(x).T @ np.abs(x)) + 1e-300
    assert np.all(np.abs(g - ref) <= tol)
    assert np.array_equal(g, g.T)


def test_gram_exact_on_integers(rq):
    x = synth.integer_matrix(3000, 70, 5)
    assert np.array_equal(host(rq.rclupp_gram(dev(x))), oracle.gram(x))


def test_gram_unit_lower(rq):
    x = synth.svd_matrix(2000, 40, 1e3, 9)
    lu, _, _, _ = oracle.gepp(x)
    M = oracle.unit_lower(lu)
    g = host(rq.rclupp_gram(dev(lu), unit_lower=True))
    ref = oracle.gram(M)
    assert np.all(np.abs(g - ref) <= 2 * gamma(2000) * (np.abs(M).T @ np.abs(M)))


@pytest.mark.parametrize("m,n", [(1, 1), (50, 3), (1000, 16), (4097, 64), (5000, 100), (3001, 129),
                                 (2100, 256)])
def test_trsm_gram(rq, m, n):
    g = np.random.default_rng(m * n)
    r = np.triu(g.standard_normal((n, n))) / math.sqrt(n) + 2 * np.eye(n)
    x = g.standard_normal((m, n))
    q, G = rq.rclupp_trsm_gram(dev(x), dev(r))
    q, G = host(q), host(G)
    q_ref = oracle.trsm(x, r)
    kap = np.linalg.cond(r)
    assert np.linalg.norm(q - q_ref) <= 10 * n * U * kap * np.linalg.norm(q_ref)
    g_ref = oracle.gram(q_ref)
    assert np.all(np.abs(G - g_ref) <= 2 * gamma(m) * (np.abs(q_ref).T @ np.abs(q_ref))
                  + 10 * n * U * kap * np.abs(g_ref).max())


def test_trsm_exact_on_unit_integer_factor(rq):
    g = np.random.default_rng(1)
    n, m = 48, 3000
    r = np.triu(g.integers(-3, 4, size=(n, n)), 1).astype(np.float64) + np.diag(g.choice([-1.0, 1.0], n))
    q0 = g.integers(-5, 6, size=(m, n)).astype(np.float64)
    x = (q0.astype(np.int64) @ r.astype(np.int64)).astype(np.float64)
    q, _ = rq.rclupp_trsm_gram(dev(x), dev(r), gram=False)
    assert np.array_equal(host(q), q0)


def test_trsm_in_place_and_padded_ld(rq):
    m, n = 3001, 33
    g = np.random.default_rng(2)
    r = np.triu(g.standard_normal((n, n))) + 3 * np.eye(n)
    x = g.standard_normal((m, n))
    # leading dimension 3005 (odd: plain-load path) and 3008 (TMA path), in place
    for ld in (3005, 3008):
        buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
        X = buf.t()[:m]
        X.copy_(dev(x))
        rq.rclupp_trsm_gram(X, dev(r), Q=X, gram=False)
        assert np.linalg.norm(host(X) - oracle.trsm(x, r)) <= 1e-12 * np.linalg.norm(host(X))
        assert float(buf.t()[m:].abs().max()) == 0.0  # rows past m untouched


# ----------------------------------------------------- small factorizations ---

@pytest.mark.parametrize("n", [1, 2, 17, 64, 128, 256])
def test_cholesky(rq, n):
    a = synth.svd_matrix(2 * n + 5, n, 1e3, n)
    gm = a.T @ a
    r, st, _ = rq.rclupp_cholesky(dev(gm))
    r_ref, _, _ = oracle.cholesky(gm)
    r = host(r)
    assert np.array_equal(r, np.triu(r))
    assert np.linalg.norm(r - r_ref) <= 10 * n * U * 1e6 * np.linalg.norm(r_ref)


def test_cholesky_exact_integer_factor(rq):
    g = np.random.default_rng(3)
    n = 20
    r0 = np.triu(g.integers(-4, 5, size=(n, n)), 1).astype(np.float64) + np.diag(g.integers(1, 5, n).astype(np.float64))
    gm = (r0.T.astype(np.int64) @ r0.astype(np.int64)).astype(np.float64)
    r, st, _ = rq.rclupp_cholesky(dev(gm))
    assert np.array_equal(host(r), r0)


def test_cholesky_breakdown_matches_oracle(rq):
    gm = np.diag([4.0, 1.0, -1.0, 2.0])
    _, st, col = rq.rclupp_cholesky(dev(gm), check=False)
    _, st_o, col_o = oracle.cholesky(gm, raise_on_error=False)
    assert st == st_o == rq.Status.ERR_CHOL_BREAKDOWN and col == col_o == 2


def test_trmm_exact(rq):
    g = np.random.default_rng(4)
    n = 77
    a = np.triu(g.integers(-5, 6, size=(n, n))).astype(np.float64)
    b = np.triu(g.integers(-5, 6, size=(n, n))).astype(np.float64)
    assert np.array_equal(host(rq.rclupp_trmm_upper(dev(a), dev(b))), oracle.trmm_upper(a, b))


@pytest.mark.parametrize("s,n", [(1, 1), (8, 3), (40, 17), (128, 64), (256, 128), (512, 256)])
def test_householder_r(rq, s, n):
    a = np.random.default_rng(s).standard_normal((s, n))
    r = host(rq.rclupp_householder_r(dev(a)))
    r_ref = oracle.householder_r(a)
    assert np.linalg.norm(r - r_ref) <= 100 * s * U * np.linalg.cond(a) * np.linalg.norm(r_ref)


@pytest.mark.parametrize("s,n,kappa", [(4, 2, 10.0), (64, 32, 1e4), (256, 128, 1e8), (300, 150, 1e2)])
def test_sketch_precond(rq, s, n, kappa):
    y = synth.svd_matrix(s, n, kappa, s)
    r1 = host(rq.rclupp_sketch_precond(dev(y)))
    r1_ref, _, _ = oracle.sketch_precond(y)
    assert np.all(np.diag(r1) > 0) and np.array_equal(r1, np.triu(r1))
    assert np.linalg.norm(r1 - r1_ref) <= 1000 * n * U * kappa * np.linalg.norm(r1_ref)


# ---------------------------------------------------------------- tall LU ---

@pytest.mark.parametrize("m,n", [(1, 1), (9, 4), (100, 16), (1000, 33), (5003, 64), (20000, 128)])
def test_tall_lupp(rq, m, n):
    x = synth.svd_matrix(m, n, 1e5, m + 7)
    lu, ipiv, st, _ = rq.rclupp_tall_lupp(dev(x))
    lu_ref, ipiv_ref, st_ref, _ = oracle.gepp(x)
    assert st == st_ref == 0
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_ref)   # pivot rows: bit-exact
    lu = host(lu)
    mm, nn = oracle.unit_lower(lu), oracle.upper(lu)
    assert np.max(np.abs(mm)) <= 1.0
    assert np.linalg.norm(lu - lu_ref) <= 1e-10 * np.linalg.norm(lu_ref)


def test_tall_lupp_integer_brute_force(rq):
    x = synth.integer_matrix(40, 8, 21, lo=-7, hi=7)
    lu, ipiv, st, _ = rq.rclupp_tall_lupp(dev(x))
    _, ipiv_ref, _, _ = oracle.gepp(x)
    assert np.array_equal(ipiv.cpu().numpy(), ipiv_ref)


def test_tall_lupp_tie_break_smallest_index(rq):
    m, n = 3000, 2
    x = np.zeros((m, n))
    x[:, 0] = 1.0
    x[[7, 1500, 2999], 0] = [-5.0, 5.0, 5.0]
    x[:, 1] = np.arange(m) % 13
    _, ipiv, _, _ = rq.rclupp_tall_lupp(dev(x))
    assert int(ipiv[0]) == 7


def test_tall_lupp_zero_pivot(rq):
    x = np.ones((500, 3))
    _, _, st, col = rq.rclupp_tall_lupp(dev(x), check=False)
    assert st == rq.Status.ERR_LU_ZERO_PIVOT and col == 1


# ----------------------------------------------------------- whole drivers ---

def _gate(x, q, r, q_o, r_o, kappa):
    orth, res = oracle.orthogonality(q), oracle.residual(x, q, r)
    orth_o, res_o = oracle.orthogonality(q_o), oracle.residual(x, q_o, r_o)
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert orth <= max(10 * orth_o, 1e-13), (orth, orth_o)
    assert res <= max(10 * res_o, 1e-13), (res, res_o)
    if kappa <= 1e6:
        assert np.linalg.norm(r - r_o) / np.linalg.norm(r_o) <= 1e-10 * kappa


DRIVERS = ["rclupp", "rcluppr", "cholqr2", "lc2"]


def _run(rq, name, x, S):
    X = dev(x)
    if name == "rclupp":
        Q, R, info = rq.rclupp_factor(X, s=S.shape[0], S=dev(S))
        q_o, r_o, _ = oracle.rclupp(x, S=S)
    elif name == "rcluppr":
        Q, R, info = rq.rclupp_r_factor(X, s=S.shape[0], S=dev(S))
        q_o, r_o, _ = oracle.rcluppr(x, S=S)
    elif name == "cholqr2":
        Q, R, info = rq.cholqr2_factor(X)
        q_o, r_o, _ = oracle.cholqr2(x)
    else:
        Q, R, info = rq.lc2_factor(X)
        q_o, r_o, _ = oracle.lc2(x)
    return host(Q), host(R), q_o, r_o


@pytest.mark.parametrize("name", DRIVERS)
@pytest.mark.parametrize("m,n,kappa", [(1, 1, 1.0), (10, 3, 10.0), (1000, 17, 1e4), (4096, 64, 1e6),
                                       (5003, 100, 1e3), (3001, 129, 1e5), (2500, 200, 1e2),
                                       (4100, 256, 1e4)])
def test_driver_parity(rq, name, m, n, kappa):
    x = synth.svd_matrix(m, n, kappa, 31 * m + n)
    S = synth.gaussian_sketch(max(2 * n, 1), m, 77)
    q, r, q_o, r_o = _run(rq, name, x, S)
    _gate(x, q, r, q_o, r_o, kappa)


@pytest.mark.parametrize("name", ["rclupp", "rcluppr", "lc2"])
@pytest.mark.parametrize("kappa", [1e8, 1e12])
def test_driver_parity_ill_conditioned(rq, name, kappa):
    m, n = 4096, 64
    x = synth.svd_matrix(m, n, kappa, 5)
    S = synth.gaussian_sketch(128, m, 6)
    q, r, q_o, r_o = _run(rq, name, x, S)
    _gate(x, q, r, q_o, r_o, kappa)


def test_cholqr2_breaks_down_like_the_oracle(rq):
    x = synth.svd_matrix(4096, 32, 1e12, 62)
    _, _, info = rq.cholqr2_factor(dev(x), check=False)
    _, _, st_o = oracle.cholqr2(x, raise_on_error=False)
    assert info.status == st_o == rq.Status.ERR_CHOL_BREAKDOWN
    assert info.failed_step in (3, 4)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("algo", ["rclupp", "rcluppr"])
def test_generated_sketch_drivers(rq, kind, algo):
    m, n, s = 8000, 64, 128
    x = synth.svd_matrix(m, n, 1e10, 44)
    fn = rq.rclupp_factor if algo == "rclupp" else rq.rclupp_r_factor
    Q, R, _ = fn(dev(x), s=s, kind=kind, zeta=8, seed=99)
    if kind == 0:
        S = oracle.gaussian_sketch_matrix(s, m, 99)
        q_o, r_o, _ = getattr(oracle, algo)(x, S=S)
    else:
        rows, signs = oracle.sparse_sign_pattern(s, m, 8, 99)
        q_o, r_o, _ = getattr(oracle, algo)(x, sparse=(s, 8, rows, signs))
    _gate(x, host(Q), host(R), q_o, r_o, 1e10)


def test_alias_q_equals_x(rq):
    m, n = 3000, 40
    x = synth.svd_matrix(m, n, 1e6, 3)
    S = synth.gaussian_sketch(80, m, 2)
    q_o, r_o, _ = oracle.rclupp(x, S=S)
    for fn in (rq.rclupp_factor, rq.rclupp_r_factor):
        X = dev(x)
        Q, R, _ = fn(X, s=80, S=dev(S), Q=X)
        _gate(x, host(X), host(R), q_o, r_o, 1e6)
    for fn in (rq.cholqr2_factor, rq.lc2_factor):
        X = dev(x)
        fn(X, Q=X)
        assert oracle.orthogonality(host(X)) < 1e-13


def test_paper_matrices_section_5_1(rq):
    # arrowhead (5.1.3) and stacked lower-triangular (5.1.2) inputs
    for x in (synth.arrowhead(1e-10, m=2000, n=20), synth.stacked_lower(-0.8, copies=40, nb=20)):
        S = synth.gaussian_sketch(40, x.shape[0], 3)
        q, r, q_o, r_o = _run(rq, "rcluppr", x, S)
        _gate(x, q, r, q_o, r_o, 1e12)


def test_argument_errors(rq):
    x = dev(np.ones((10, 4)))
    with pytest.raises(rq.RclupError) as e:
        rq.rclupp_factor(x, s=2)  # s < n
    assert e.value.status == rq.Status.ERR_ARG
    with pytest.raises(rq.RclupError) as e:
        rq.cholqr2_factor(dev(np.ones((3, 5))))  # m < n
    assert e.value.status == rq.Status.ERR_ARG
    with pytest.raises(rq.RclupError) as e:
        rq.rclupp_factor(dev(np.ones((600, 300))))  # n > 256
    assert e.value.status == rq.Status.ERR_UNSUPPORTED


def test_deterministic_repeat(rq):
    x = synth.svd_matrix(20000, 64, 1e6, 12)
    X = dev(x)
    Q1, R1, _ = rq.rclupp_factor(X, s=128, seed=5)
    Q2, R2, _ = rq.rclupp_factor(X, s=128, seed=5)
    assert torch.equal(Q1, Q2) and torch.equal(R1, R2)
