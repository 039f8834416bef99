"""Binary64-emulating tensor-core Gram (split-bf16 digits, exact fp32 level
sums) and the RCLUPP_PREC_EMULATED tier of the drivers, against the oracle.

Error model of the emulated Gram G = A^T A.  With E_j the column exponent
(2^E_j > max_i |a_ij|), the digit split rounds a_ij at 2^(E_j - 64) and the
product keeps the levels s + t <= 7 of the 8 x 8 digit products; both
perturb G(j, k) by far less than m 2^-53 2^(E_j + E_k).  The fp32 window
sums are exact, the int64 drain rounds levels 5..7 (2^-50 of a window's
scale) and the binary64 combination adds at most (m / 128 + 2) u |A|^T |A|.
The tests bound the distance to the exact Gram (Python integers on
integer-scaled inputs) or to the binary64 oracle (whose own error is
gamma_m |A|^T |A|) with the binary64-like bound 4 (m + 128) u 2^(E_j + E_k).
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
    a = np.asfortranarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda").t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


@pytest.fixture(scope="module")
def rq():
    import paper_2412_06551_gb300 as m
    m.load()
    return m


def col_scale(x):
    """2^E_j with 2^E_j > max_i |x_ij| (the smallest such power of two)."""
    mx = np.max(np.abs(x), axis=0)
    e = np.where(mx > 0, np.floor(np.log2(np.where(mx > 0, mx, 1.0))) + 1, -1022)
    return np.ldexp(1.0, e.astype(int))


def emu_bound(x):
    m = x.shape[0]
    sc = col_scale(x)
    a = np.abs(x)
    return 4 * (m + 128) * U * np.outer(sc, sc) + (m / 128 + 2) * U * (a.T @ a)


def test_exact_on_small_integers(rq):
    # |x| <= 100: one digit per entry, every level sum exact -> G exact
    g = np.random.default_rng(1)
    for m, n in [(1, 1), (300, 7), (5000, 64), (2049, 128), (1500, 200), (777, 256)]:
        x = g.integers(-100, 101, size=(m, n)).astype(np.float64)
        G = host(rq.rclupp_gram_emulated(dev(x)))
        xi = x.astype(np.int64)
        assert np.array_equal(G, (xi.T @ xi).astype(np.float64)), (m, n)


def test_all_digits_against_exact_integers(rq):
    # x = k 2^-40 with |k| < 2^47: the scaled value k 2^(63 - E - 40) is an
    # exact integer, so all digits are used and the only errors are the
    # dropped levels and the drain and binary64 combination; the exact Gram
    # comes from Python integers
    g = np.random.default_rng(2)
    for m, n in [(129, 5), (1000, 48), (3001, 130)]:
        k = g.integers(-(2 ** 46), 2 ** 46, size=(m, n), dtype=np.int64)
        x = np.ldexp(k.astype(np.float64), -40)
        assert np.array_equal(np.ldexp(x, 40).astype(np.int64), k)  # exact
        G = host(rq.rclupp_gram_emulated(dev(x)))
        ko = k.astype(object)
        exact = ko.T.dot(ko)
        ref = np.array([[math.ldexp(float(v), -80) for v in row] for row in exact])
        err = np.abs(G - ref)
        assert np.all(err <= emu_bound(x)), float(np.max(err / emu_bound(x)))


@pytest.mark.parametrize("m,n", [(1, 1), (127, 3), (128, 64), (129, 65), (1000, 100), (5000, 128),
                                 (3001, 129), (2100, 256), (70001, 200), (262144, 128)])
def test_against_oracle(rq, m, n):
    g = np.random.default_rng(m + n)
    x = g.standard_normal((m, n)) * np.logspace(-3, 3, n)  # columns of very different scales
    G = host(rq.rclupp_gram_emulated(dev(x)))
    ref = oracle.gram(x)
    a = np.abs(x)
    tol = emu_bound(x) + gamma(m) * (a.T @ a)
    assert np.all(np.abs(G - ref) <= tol), float(np.max(np.abs(G - ref) / tol))
    assert np.array_equal(G, G.T)


def test_special_columns(rq):
    m, n = 3000, 6
    g = np.random.default_rng(3)
    x = g.standard_normal((m, n))
    x[:, 1] = 0.0                      # zero column
    x[:, 2] *= 1e-310                  # subnormal entries
    x[:, 3] *= 1e150                   # large scale (x^2 ~ 1e300 is finite)
    G = host(rq.rclupp_gram_emulated(dev(x)))
    ref = oracle.gram(x)
    assert np.all(G[1, :] == 0) and np.all(G[:, 1] == 0)
    ok = np.ones((n, n), bool)
    ok[1, :] = ok[:, 1] = False
    a = np.abs(x)
    tol = emu_bound(x) + gamma(m) * (a.T @ a)
    assert np.all(np.abs(G - ref)[ok] <= tol[ok])
    x[5, 4] = np.nan                   # a non-finite column poisons its row/column only
    G = host(rq.rclupp_gram_emulated(dev(x)))
    assert np.all(np.isnan(G[4, :])) and np.all(np.isnan(G[:, 4]))
    assert np.all(np.isfinite(np.delete(np.delete(G, 4, 0), 4, 1)))


def test_deterministic_and_ld(rq):
    m, n = 40000, 96
    x = synth.svd_matrix(m, n, 1e6, 5)
    X = dev(x)
    assert torch.equal(rq.rclupp_gram_emulated(X), rq.rclupp_gram_emulated(X))
    buf = torch.zeros((n, m + 3), dtype=torch.float64, device="cuda")
    Xp = buf.t()[:m]
    Xp.copy_(X)
    assert torch.equal(rq.rclupp_gram_emulated(Xp), rq.rclupp_gram_emulated(X))


def _gate(x, q, r, q_o, r_o, kappa):
    orth, res = oracle.orthogonality(q), oracle.residual(x, q, r)
    orth_o, res_o = oracle.orthogonality(q_o), oracle.residual(x, q_o, r_o)
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert orth <= max(10 * orth_o, 1e-13), (orth, orth_o)
    assert res <= max(10 * res_o, 1e-13), (res, res_o)
    if kappa <= 1e6:
        assert np.linalg.norm(r - r_o) / np.linalg.norm(r_o) <= 1e-10 * kappa


@pytest.mark.parametrize("algo", ["rclupp", "rcluppr"])
@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10, 1e12])
@pytest.mark.parametrize("tier", [3, 4])
def test_driver_emulated_tier(rq, algo, kappa, tier):
    m, n, s = 8192, 64, 128
    x = synth.svd_matrix(m, n, kappa, 81)
    fn = rq.rclupp_factor if algo == "rclupp" else rq.rclupp_r_factor
    Q, R, info = fn(dev(x), s=s, seed=7, prec=tier)
    q_o, r_o, _ = getattr(oracle, algo)(x, S=oracle.gaussian_sketch_matrix(s, m, 7))
    _gate(x, host(Q), host(R), q_o, r_o, kappa)
    assert info.emulated == tier - 2
    assert info.prec_used == rq.PREC_SKETCH_DIGITS  # the emulated tiers' sketch, never escalated


@pytest.mark.parametrize("m,n,kappa", [(20000, 128, 1e4), (9000, 256, 1e8)])
def test_all_emulated_explicit_sketch(rq, m, n, kappa):
    x = synth.svd_matrix(m, n, kappa, 90 + n)
    S = synth.gaussian_sketch(2 * n, m, 17)
    Q, R, info = rq.rclupp_factor(dev(x), s=2 * n, S=dev(S), prec=rq.PREC_EMULATED_ALL)
    q_o, r_o, _ = oracle.rclupp(x, S=S)
    _gate(x, host(Q), host(R), q_o, r_o, kappa)
    assert info.emulated == 2 and info.prec_used == 0
    Q2, R2, info2 = rq.rcholqr_factor(dev(x), s=2 * n, S=dev(S), prec=rq.PREC_EMULATED_ALL)
    q2, r2, _ = oracle.rcholqr(x, S=S)
    _gate(x, host(Q2), host(R2), q2, r2, kappa)


@pytest.mark.parametrize("m,n,kappa", [(4096, 64, 1e8), (5003, 128, 1e4), (3000, 256, 1e3),
                                       (1000, 17, 1e10)])
def test_emulated_with_explicit_sketch(rq, m, n, kappa):
    # explicit S: binary64 sketch, emulated first-pass Gram; same S as the oracle
    x = synth.svd_matrix(m, n, kappa, 82 + n)
    S = synth.gaussian_sketch(2 * n, m, 13)
    Q, R, info = rq.rclupp_factor(dev(x), s=2 * n, S=dev(S), prec=rq.PREC_EMULATED)
    q_o, r_o, _ = oracle.rclupp(x, S=S)
    _gate(x, host(Q), host(R), q_o, r_o, kappa)
    assert info.emulated == 1 and info.prec_used == 0
    Q2, R2, info2 = rq.rcholqr_factor(dev(x), s=2 * n, S=dev(S), prec=rq.PREC_EMULATED)
    q2, r2, _ = oracle.rcholqr(x, S=S)
    if kappa <= 1e8:
        _gate(x, host(Q2), host(R2), q2, r2, kappa)
    assert info2.emulated == 1


# ---------------------------------------------------------------- triangular solve ---

def trsm_bound(x, r, q_ref):
    """|Q_emu - Q_ref| bound: the emulated updates perturb C_J by about
    (n + 128) 2^-53 2^(E_i + E'_c) per entry; substitution turns a
    perturbation of A into one of Q through R^{-1}; plus both sides' binary64
    rounding (n u kappa-like growth, taken from |Q| |R| |R^{-1}|)."""
    m, n = x.shape
    qs = col_scale(np.abs(q_ref).T).reshape(-1, 1)  # per-row scale of Q
    rs = col_scale(r)                               # per-column scale of R
    rinv = np.abs(np.linalg.inv(r))
    pert = (n + 128) * 4 * U * (qs * (np.ones((1, n)) * rs.max())) * n
    return pert @ rinv + 20 * n * U * (np.abs(q_ref) @ np.abs(r)) @ rinv


@pytest.mark.parametrize("m,n", [(1, 1), (300, 31), (1000, 32), (3001, 33), (5000, 64), (4097, 100),
                                 (2048, 128), (3000, 129), (2100, 256), (70001, 200)])
def test_trsm_emulated_against_oracle(rq, m, n):
    g = np.random.default_rng(m * n + 1)
    r = np.triu(g.standard_normal((n, n))) / math.sqrt(n) + 2 * np.eye(n)
    x = g.standard_normal((m, n)) * np.logspace(-2, 2, n)
    q = host(rq.rclupp_trsm_emulated(dev(x), dev(r)))
    q_ref = oracle.trsm(x, r)
    err = np.abs(q - q_ref)
    tol = trsm_bound(x, r, q_ref)
    assert np.all(err <= tol), float(np.max(err / tol))
    # residual of the solve at binary64 level
    assert np.linalg.norm(q @ r - x) <= 50 * n * U * np.linalg.norm(np.abs(q) @ np.abs(r))


def test_trsm_emulated_exact_on_integers(rq):
    # unit upper R with small integers and Q0 with small integers: every update
    # is an exact integer of few digits, so Q comes back exactly
    g = np.random.default_rng(4)
    for n, m in [(48, 3000), (130, 1000), (256, 700)]:
        r = np.triu(g.integers(-3, 4, size=(n, n)), 1).astype(np.float64) + np.diag(g.choice([-1.0, 1.0], n))
        q0 = g.integers(-5, 6, size=(m, n)).astype(np.float64)
        x = (q0.astype(np.int64) @ r.astype(np.int64)).astype(np.float64)
        assert np.max(np.abs(x)) < 2 ** 50
        q = host(rq.rclupp_trsm_emulated(dev(x), dev(r)))
        assert np.array_equal(q, q0), (n, m)


def test_trsm_emulated_in_place_and_ld(rq):
    m, n = 3001, 97
    g = np.random.default_rng(5)
    r = np.triu(g.standard_normal((n, n))) + 3 * np.eye(n)
    x = g.standard_normal((m, n))
    ref = host(rq.rclupp_trsm_emulated(dev(x), dev(r)))
    for ld in (3005, 3008):
        buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
        X = buf.t()[:m]
        X.copy_(dev(x))
        rq.rclupp_trsm_emulated(X, dev(r), Q=X)
        assert np.array_equal(host(X), ref)
        assert float(buf.t()[m:].abs().max()) == 0.0


# ------------------------------- solve by a well-conditioned factor (C3, C7) ---

def _wellcond_r(n, seed, spread=0.1):
    g = np.random.default_rng(seed)
    return np.eye(n) + spread * np.triu(g.standard_normal((n, n)), 1) / math.sqrt(n)


@pytest.mark.parametrize("m,n", [(1, 1), (300, 31), (5000, 64), (4097, 100), (2048, 128), (3001, 129),
                                 (2100, 256), (70001, 200)])
def test_wellcond_solve_product_against_oracle(rq, m, n):
    # cond(R) ~ 1.5: the product Q = X R^{-1} runs; against the oracle's
    # substitution, both within the rounding of R^{-1} (|W| |R| |W|, the
    # triangular inverse's error) and the digits' 2^-50 of the row and column
    # maxima
    g = np.random.default_rng(m + 7 * n)
    r = _wellcond_r(n, m + n)
    x = g.standard_normal((m, n)) * np.logspace(-3, 3, m)[:, None]
    q, form = rq.rclupp_trsm_emulated_wellcond(dev(x), dev(r))
    assert form == 1
    q = host(q)
    q_ref = oracle.trsm(x, r)
    w = np.abs(np.linalg.inv(r))
    tol = (16 * n * U * (np.abs(x) @ (w @ np.abs(r) @ w))
           + (n + 128) * 2.0 ** -50 * np.max(np.abs(x), axis=1)[:, None] * np.max(w, axis=0)[None, :])
    assert np.all(np.abs(q - q_ref) <= tol), float(np.max(np.abs(q - q_ref) / tol))
    assert np.linalg.norm(q @ r - x) <= 100 * n * U * np.linalg.norm(np.abs(q) @ np.abs(r))


def test_wellcond_solve_exact_on_integers(rq):
    # R = I + superdiagonal of ones: R^{-1} has entries (-1)^(j - i) above the
    # diagonal (Skeel's cond(R) = 2n - 1 = 79), X = Q0 R with small integers: every digit
    # product and sum is exact, so Q = Q0
    n, m = 40, 3000
    r = np.eye(n) + np.diag(np.ones(n - 1), 1)
    q0 = np.random.default_rng(3).integers(-9, 10, size=(m, n)).astype(np.float64)
    x = q0 @ r
    q, form = rq.rclupp_trsm_emulated_wellcond(dev(x), dev(r))
    assert form == 1 and np.array_equal(host(q), q0)


def test_wellcond_solve_falls_back_to_substitution(rq):
    # an ill-conditioned factor (cond(R) far above max(100, n)) takes the emulated
    # substitution, bit for bit the result of rclupp_trsm_emulated
    n, m = 96, 5000
    g = np.random.default_rng(11)
    r = np.triu(g.standard_normal((n, n))) / math.sqrt(n) + np.diag(np.logspace(0, -6, n))
    x = g.standard_normal((m, n))
    q, form = rq.rclupp_trsm_emulated_wellcond(dev(x), dev(r))
    assert form == 0
    assert torch.equal(q, rq.rclupp_trsm_emulated(dev(x), dev(r)))


def test_wellcond_solve_in_place_and_nonfinite(rq):
    n, m = 150, 4001
    r = _wellcond_r(n, 5)
    x = np.random.default_rng(6).standard_normal((m, n))
    ref, form = rq.rclupp_trsm_emulated_wellcond(dev(x), dev(r))
    assert form == 1
    for ld in (4001, 4008):
        buf = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
        X = buf.t()[:m]
        X.copy_(dev(x))
        rq.rclupp_trsm_emulated_wellcond(X, dev(r), Q=X)
        assert torch.equal(X, ref)
        if ld > m:
            assert float(buf.t()[m:].abs().max()) == 0.0
    xn = x.copy()
    xn[17, 3] = np.inf
    q, _ = rq.rclupp_trsm_emulated_wellcond(dev(xn), dev(r))
    q = host(q)
    assert np.all(np.isnan(q[17])) and np.all(np.isfinite(np.delete(q, 17, axis=0)))


def _skeel(r):
    """Skeel's condition number || |R^-1| |R| ||_inf of an upper-triangular R."""
    return float(np.max(np.abs(np.linalg.inv(r)) @ np.abs(r).sum(axis=1)))


@pytest.mark.parametrize("n", [64, 128, 256])
def test_wellcond_solve_selects_by_skeel_condition_of_a_sketch_factor(rq, n):
    # R2 of the emulated tiers: the Cholesky factor of Q1^T Q1, Q1 = X R1^{-1}
    # after a Gaussian embedding with s = 2n (kappa(Q1) ~ 6).  Its 1-norm
    # condition number exceeds 100 from n = 128 on, but Skeel's condition
    # number, the factor in the product's residual bound, stays below
    # max(100, n): the product runs, and matches the oracle's substitution
    # within the bound of the product test above.
    m = 8 * n
    g = np.random.default_rng(n)
    x = synth.svd_matrix(m, n, 1e4, 40 + n)
    y = (g.standard_normal((2 * n, m)) / math.sqrt(2 * n)) @ x
    r1 = np.linalg.qr(y, mode="r")
    q1 = np.linalg.solve(r1.T, x.T).T
    r = np.linalg.cholesky(q1.T @ q1).T
    cond = _skeel(r)
    kappa_1 = np.abs(r).sum(axis=0).max() * np.abs(np.linalg.inv(r)).sum(axis=0).max()
    assert cond <= max(100.0, n)
    if n >= 128:
        assert kappa_1 > 100.0
    a = g.standard_normal((3001, n))
    q, form = rq.rclupp_trsm_emulated_wellcond(dev(a), dev(r))
    assert form == 1
    q = host(q)
    q_ref = oracle.trsm(a, r)
    w = np.abs(np.linalg.inv(r))
    tol = (16 * n * U * (np.abs(a) @ (w @ np.abs(r) @ w))
           + (n + 128) * 2.0 ** -50 * np.max(np.abs(a), axis=1)[:, None] * np.max(w, axis=0)[None, :])
    assert np.all(np.abs(q - q_ref) <= tol), float(np.max(np.abs(q - q_ref) / tol))


def test_wellcond_solve_rejects_above_the_skeel_limit(rq):
    # a factor with Skeel's condition number above max(100, n) = 100 (about
    # 214 for this unit upper-triangular R with N(0, 4/n) entries above the
    # diagonal) takes the substitution, bit for bit
    n, m = 64, 2000
    g = np.random.default_rng(21)
    r = np.eye(n) + 2.0 * np.triu(g.standard_normal((n, n)), 1) / math.sqrt(n)
    cond = _skeel(r)
    assert 150.0 < cond < 300.0, cond
    x = g.standard_normal((m, n))
    q, form = rq.rclupp_trsm_emulated_wellcond(dev(x), dev(r))
    assert form == 0
    assert torch.equal(q, rq.rclupp_trsm_emulated(dev(x), dev(r)))
