"""Parity of the subsampled randomized Hadamard sketch (SRHT, one of the
common sketches of Section 3) with the oracle's implementation of the same
definition: S(r, i) = d_i (-1)^popcount(p_r AND i) / sqrt(s), the signs and
sampled rows drawn from the same counter-based generator on both sides.

Tolerances: the oracle sums m products sequentially (within gamma_m |S||x| of
the exact value); the kernel transforms each 256-row block exactly in
integers after rounding the block's entries to 53 bits relative to its
largest (at most u max|x_block| per entry), then adds the sampled values in
binary64 (within gamma_k of their sum, k << m).  Integer-valued inputs with
s a power of four (1/sqrt(s) a power of two) are exact on both sides and are
compared bit for bit.
"""
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
    a = np.asfortranarray(a, dtype=np.float64)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda").t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


@pytest.fixture(scope="module")
def rq():
    import paper_2412_06551_gb300 as m
    m.load()
    return m


def _block_term(x, row0, s):
    """sum over 256-row blocks of 256 u max|x_block| / sqrt(s), per column."""
    m, n = x.shape
    out = np.zeros(n)
    g0 = row0 // 256
    g1 = (row0 + m - 1) // 256
    for g in range(g0, g1 + 1):
        lo, hi = max(0, g * 256 - row0), min(m, g * 256 + 256 - row0)
        out += np.abs(x[lo:hi]).max(axis=0)
    return 256 * U * out / np.sqrt(s)


def _tol(S, x, row0=0):
    m = x.shape[0]
    return (2 * gamma(m) * (np.abs(S) @ np.abs(x)) + _block_term(x, row0, S.shape[0])[None, :]
            + 1e-300)


@pytest.mark.parametrize("m,n,s,seed", [(1, 1, 1, 0), (2, 1, 2, 3), (255, 3, 8, 1), (256, 16, 64, 2),
                                        (257, 17, 33, 5), (5000, 32, 64, 0), (4096, 64, 128, 123),
                                        (3001, 40, 300, 9), (20001, 128, 256, 2 ** 40 + 5),
                                        (6000, 20, 700, 4), (9000, 9, 1500, 6), (4100, 5, 3000, 8),
                                        (8192, 2, 4096, 10)])
def test_srht_matches_oracle(rq, m, n, s, seed):
    x = synth.svd_matrix(m, n, 1e2, m + n) if m >= n else synth.integer_matrix(m, n, 1)
    y = host(rq.rclupp_sketch(dev(x), s=s, kind=rq.SKETCH_SRHT, seed=seed))
    S = oracle.srht_dense(s, m, seed)
    ref = oracle.sketch_dense(S, x)
    assert np.all(np.abs(y - ref) <= _tol(S, x))


@pytest.mark.parametrize("m,n,s", [(300, 7, 16), (1000, 16, 64), (5000, 33, 256), (4096, 3, 1024)])
def test_srht_exact_on_integers(rq, m, n, s):
    # integer X, s a power of four: every step is exact on both sides
    x = synth.integer_matrix(m, n, m + s).astype(np.float64) * 1000.0
    y = host(rq.rclupp_sketch(dev(x), s=s, kind=rq.SKETCH_SRHT, seed=s))
    root = int(round(np.sqrt(s)))
    H = np.rint(oracle.srht_dense(s, m, s) * root).astype(np.int64)
    exact = (H @ x.astype(np.int64)).astype(np.float64) / root
    assert np.array_equal(y, exact)


def test_srht_wide_dynamic_range(rq):
    # entries spanning 2^-200 .. 2^200 within blocks and across blocks
    g = np.random.default_rng(5)
    m, n, s = 3000, 6, 64
    x = g.standard_normal((m, n)) * np.exp2(g.integers(-200, 200, size=(m, n)))
    y = host(rq.rclupp_sketch(dev(x), s=s, kind=rq.SKETCH_SRHT, seed=1))
    S = oracle.srht_dense(s, m, 1)
    assert np.all(np.abs(y - oracle.sketch_dense(S, x)) <= _tol(S, x))


def test_srht_tiny_and_subnormal_blocks(rq):
    m, n, s = 700, 3, 16
    x = np.zeros((m, n))
    x[:256, 0] = 1e-310 * np.arange(1, 257)        # subnormal block
    x[256:512, 1] = np.ldexp(1.0, -1060)            # one tiny value per row
    x[600, 2] = 3.0
    y = host(rq.rclupp_sketch(dev(x), s=s, kind=rq.SKETCH_SRHT, seed=2))
    S = oracle.srht_dense(s, m, 2)
    assert np.all(np.abs(y - oracle.sketch_dense(S, x)) <= _tol(S, x))
    assert np.any(y[:, 0] != 0) and np.all(np.isfinite(y))


def test_srht_nonfinite_column_is_nan(rq):
    x = synth.svd_matrix(1000, 4, 1e2, 3)
    x[700, 2] = np.inf
    y = host(rq.rclupp_sketch(dev(x), s=32, kind=rq.SKETCH_SRHT, seed=1))
    assert np.all(np.isnan(y[:, 2]))
    S = oracle.srht_dense(32, 1000, 1)
    ok = [0, 1, 3]
    assert np.all(np.abs(y[:, ok] - oracle.sketch_dense(S, x[:, ok])) <= _tol(S, x[:, ok]))


@pytest.mark.parametrize("row0", [0, 1000, 4097])
def test_srht_row_blocks_sum_to_whole(rq, row0):
    m, n, s, seed = 9000, 12, 64, 3
    x = synth.svd_matrix(m, n, 1e3, 11)
    b = oracle.srht_order_log2(row0 + m)
    whole = host(rq.rclupp_sketch(dev(x), s=s, kind=rq.SKETCH_SRHT, seed=seed, row0=row0, order_log2=b))
    S = oracle.srht_dense(s, m, seed, b=b, row0=row0)
    assert np.all(np.abs(whole - oracle.sketch_dense(S, x)) <= _tol(S, x, row0))
    cut = 3333
    y1 = host(rq.rclupp_sketch(dev(x[:cut]), s=s, kind=rq.SKETCH_SRHT, seed=seed, row0=row0,
                               order_log2=b))
    y2 = host(rq.rclupp_sketch(dev(x[cut:]), s=s, kind=rq.SKETCH_SRHT, seed=seed, row0=row0 + cut,
                               order_log2=b))
    assert np.all(np.abs(y1 + y2 - whole) <= 2 * _tol(S, x, row0))


def test_srht_explicit_order(rq):
    m, n, s = 1000, 8, 40
    x = synth.svd_matrix(m, n, 1e2, 12)
    y = host(rq.rclupp_sketch(dev(x), s=s, kind=rq.SKETCH_SRHT, seed=7, order_log2=14))
    S = oracle.srht_dense(s, m, 7, b=14)
    assert np.all(np.abs(y - oracle.sketch_dense(S, x)) <= _tol(S, x))


def test_srht_unit_lower_factor(rq):
    m, n, s = 3000, 24, 48
    x = synth.svd_matrix(m, n, 1e4, 8)
    lu, ipiv, st, _ = oracle.gepp(x)
    M = oracle.unit_lower(lu)
    y = host(rq.rclupp_sketch(dev(lu), s=s, kind=rq.SKETCH_SRHT, seed=4, unit_lower=True))
    S = oracle.srht_dense(s, m, 4)
    assert np.all(np.abs(y - oracle.sketch_dense(S, M)) <= _tol(S, M))


def test_srht_deterministic_and_padded_ld(rq):
    m, n, s = 5000, 20, 100
    x = synth.svd_matrix(m, n, 1e2, 13)
    X = dev(x)
    y1 = rq.rclupp_sketch(X, s=s, kind=rq.SKETCH_SRHT, seed=9)
    y2 = rq.rclupp_sketch(X, s=s, kind=rq.SKETCH_SRHT, seed=9)
    assert torch.equal(y1, y2)
    big = torch.zeros((n, m + 37), dtype=torch.float64, device="cuda").t()
    big[:m] = X
    y3 = rq.rclupp_sketch(big[:m], s=s, kind=rq.SKETCH_SRHT, seed=9)
    assert torch.equal(y1, y3)


def test_srht_argument_errors(rq):
    x = dev(synth.svd_matrix(100, 4, 10.0, 1))
    with pytest.raises(rq.RclupError) as e:  # s = 200 > 2^7
        rq.rclupp_sketch(x, s=200, kind=rq.SKETCH_SRHT)
    assert e.value.status == rq.Status.ERR_ARG
    with pytest.raises(rq.RclupError) as e:  # order 2^6 < m
        rq.rclupp_sketch(x, s=8, kind=rq.SKETCH_SRHT, order_log2=6)
    assert e.value.status == rq.Status.ERR_ARG
    y = host(rq.rclupp_sketch(x, s=200, kind=rq.SKETCH_SRHT, order_log2=8))
    assert y.shape == (200, 4) and np.all(np.isfinite(y))


# --------------------------------------------------------------- drivers ---

def _gate(x, q, r, q_o, r_o, kappa):
    orth, res = oracle.orthogonality(q), oracle.residual(x, q, r)
    orth_o, res_o = oracle.orthogonality(q_o), oracle.residual(x, q_o, r_o)
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert orth <= max(10 * orth_o, 1e-13), (orth, orth_o)
    assert res <= max(10 * res_o, 1e-13), (res, res_o)
    if kappa <= 1e6:
        assert np.linalg.norm(r - r_o) / np.linalg.norm(r_o) <= 1e-10 * kappa


@pytest.mark.parametrize("algo", ["rclupp", "rcluppr", "rcholqr"])
@pytest.mark.parametrize("kappa", [1e4, 1e10])
def test_srht_drivers_match_oracle(rq, algo, kappa):
    m, n, s = 8000, 64, 128
    if algo == "rcholqr" and kappa > 1e6:
        kappa = 1e6  # one sketch + one CholeskyQR (Algorithm 5) needs kappa well below 1/u
    x = synth.svd_matrix(m, n, kappa, 45)
    fn = {"rclupp": rq.rclupp_factor, "rcluppr": rq.rclupp_r_factor, "rcholqr": rq.rcholqr_factor}[algo]
    Q, R, info = fn(dev(x), s=s, kind=rq.SKETCH_SRHT, seed=99)
    S = oracle.srht_dense(s, m, 99)
    q_o, r_o, _ = getattr(oracle, algo)(x, S=S)
    _gate(x, host(Q), host(R), q_o, r_o, kappa)
    assert info.prec_used == rq.PREC_FP64


@pytest.mark.parametrize("prec", [1, 3, 4])
def test_srht_keeps_binary64_sketch_at_every_tier(rq, prec):
    m, n, s = 6000, 48, 96
    x = synth.svd_matrix(m, n, 1e8, 46)
    Q, R, info = rq.rclupp_factor(dev(x), s=s, kind=rq.SKETCH_SRHT, seed=5, prec=prec)
    assert info.prec_used == rq.PREC_FP64
    assert info.emulated == (prec - 2 if prec >= 3 else 0)
    q_o, r_o, _ = oracle.rclupp(x, S=oracle.srht_dense(s, m, 5))
    _gate(x, host(Q), host(R), q_o, r_o, 1e8)


def test_srht_batched_matches_single_calls(rq):
    g = np.random.default_rng(6)
    xs = [synth.svd_matrix(int(mm), int(nn), 1e6, 900 + i)
          for i, (mm, nn) in enumerate(zip(g.integers(300, 5000, 8), g.choice([8, 33, 64, 100], 8)))]
    Xs = [dev(x) for x in xs]
    Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=rq.ALGO_RCLUPP, seed=31, kind=rq.SKETCH_SRHT)
    assert np.all(st == 0)
    for i, X in enumerate(Xs):
        q, r, _ = rq.rclupp_factor(X, s=2 * X.shape[1], seed=31 + i, kind=rq.SKETCH_SRHT)
        assert torch.equal(Qb[i], q) and torch.equal(Rb[i], r), i


# ------------------------------------------------------------- full size ---

@pytest.mark.slow
def test_srht_full_size_m1M_n128(rq):
    """m = 2^20, n = 128, s = 256 (the side-by-side workload's shape): sampled
    rows of S X recomputed by the oracle, and RCLUPP with the SRHT against
    the unique positive-diagonal R of the Gaussian-sketch factorization."""
    m, n, s, seed = 1 << 20, 128, 256, 17
    x = synth.svd_matrix(m, n, 1e4, synth.kappa_seed(1, 0))
    X = dev(x)
    y = host(rq.rclupp_sketch(X, s=s, kind=rq.SKETCH_SRHT, seed=seed))
    rows = [0, 1, 77, 128, 255]
    Srows = oracle.srht_dense_rows(rows, s, m, seed)
    ref = oracle.sketch_dense(Srows, x)
    tol = 2 * gamma(m) * (np.abs(Srows) @ np.abs(x)) + _block_term(x, 0, s)[None, :]
    assert np.all(np.abs(y[rows] - ref) <= tol)
    Q, R, info = rq.rclupp_factor(X, s=s, kind=rq.SKETCH_SRHT, seed=seed)
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert float(torch.linalg.norm(Q.t() @ Q - eye)) <= 1e-13
    assert float(torch.linalg.norm(Q @ R - X) / torch.linalg.norm(X)) <= 1e-13
    _, Rg, _ = rq.rclupp_factor(X, s=s, seed=seed)
    r, rg = host(R), host(Rg)
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert np.linalg.norm(r - rg) / np.linalg.norm(rg) <= 1e-10 * 1e4
