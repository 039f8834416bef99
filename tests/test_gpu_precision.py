"""Reduced-precision sketch tier (tensor cores) against the oracle.

The tensor-core sketch computes Y = z_b X_split / sqrt(s) with fp32 sums
inside each CTA and binary64 sums across CTAs, z_b the bf16 levels of a
discretised normal drawn by Philox.  The oracle evaluates the same
definition (levels, one- or three-term bf16 split of X) in binary64; every
product is exact in fp32, so the two differ only by the fp32 summation:
|Y_gpu - Y_ref| <= gamma32_m (|z_b| |X_split|) / sqrt(s) with
gamma32_k = k 2^-24 / (1 - k 2^-24), and |X_split| <= (1 + 2^-7) |X|.
A sketch of unit columns has one product per entry, so it reproduces S
itself bit for bit: that pins the device's level table and draw.

The drivers must meet the same gates as the binary64 path against the
binary64 oracle, reporting the tier that produced the result.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def gamma32(k):
    u = 2.0 ** -24
    return k * u / (1 - k * u)


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


@pytest.mark.parametrize("prec,nterms", [(1, 1), (2, 3)])
@pytest.mark.parametrize("m,n,s", [(1, 1, 1), (100, 7, 8), (4096, 64, 128), (5003, 128, 256),
                                   (3001, 200, 300), (2048, 256, 512), (20001, 16, 32)])
def test_tc_sketch_matches_definition(rq, prec, nterms, m, n, s):
    x = synth.svd_matrix(m, n, 1e3, m + n) if m >= n else synth.integer_matrix(m, n, 1)
    seed = 1234 + m
    y = host(rq.rclupp_sketch(dev(x), s=s, seed=seed, prec=prec))
    ref = oracle.sketch_bf16(s, seed, nterms, x)
    S = oracle.tier_sketch_z(s, m, seed) / np.sqrt(s)  # z_b / sqrt(s) in binary64
    mag = (1 + 2.0 ** -7) * (np.abs(S) @ np.abs(x))
    assert np.all(np.abs(y - ref) <= gamma32(m) * mag + 1e-300)
    # and close to the same S times the unrounded X: X's rounding (2^-9 for
    # one term, 2^-23 for three) plus the fp32 sums
    full = oracle.sketch_dense(S, x)
    rel = np.max(np.abs(y - full) / (mag + 1e-300))
    assert rel <= (2.0 ** -9 if nterms == 1 else 2.0 ** -23) + gamma32(m)


@pytest.mark.parametrize("prec", [1, 2])
def test_tc_sketch_of_unit_columns_is_s_itself(rq, prec):
    # Y = S [e_0 .. e_255]: one product per entry, exact in fp32, so Y holds
    # 512 x 256 entries of S bit for bit -- about 32 draws of each of the 4096
    # table entries, so every level of the device's table is compared
    m, s, seed = 256, 512, 99
    y = host(rq.rclupp_sketch(dev(np.eye(m)), s=s, seed=seed, prec=prec))
    assert np.array_equal(y, oracle.sketch_bf16(s, seed, 1, np.eye(m)))
    z = oracle.tier_sketch_z(s, m, seed)
    assert set(np.unique(z)) == set(np.unique(oracle.tier_levels()))


@pytest.mark.parametrize("row0", [0, 3, 8, 13])
def test_tc_sketch_row_block_draws_the_global_entries(rq, row0):
    # a row block starting at global row row0 (not necessarily a multiple of
    # the 8 entries one Philox block gives) uses the entries (r, row0 + i)
    m, n, s, seed = 300, 5, 64, 17
    x = synth.integer_matrix(m, n, row0 + 1)
    y = host(rq.rclupp_sketch(dev(x), s=s, seed=seed, prec=1, row0=row0))
    z = oracle.tier_sketch_z(s, row0 + m, seed)[:, row0:]
    assert np.array_equal(y, (z @ x) * (1.0 / np.sqrt(s)))


def test_tc_sketch_unit_lower(rq):
    m, n, s = 3000, 24, 48
    x = synth.svd_matrix(m, n, 1e4, 8)
    lu, _, _, _ = oracle.gepp(x)
    M = oracle.unit_lower(lu)
    y = host(rq.rclupp_sketch(dev(lu), s=s, seed=4, prec=2, unit_lower=True))
    ref = oracle.sketch_bf16(s, 4, 3, M)
    S = oracle.tier_sketch_z(s, m, 4) / np.sqrt(s)
    mag = 1.02 * (np.abs(S) @ np.abs(M))
    assert np.all(np.abs(y - ref) <= gamma32(m) * mag + 1e-300)


def test_tc_sketch_deterministic(rq):
    x = synth.svd_matrix(50000, 128, 1e2, 3)
    X = dev(x)
    y1 = rq.rclupp_sketch(X, s=256, seed=9, prec=2)
    y2 = rq.rclupp_sketch(X, s=256, seed=9, prec=2)
    assert torch.equal(y1, y2)


def _gate(x, q, r, q_o, r_o, kappa):
    orth, res = oracle.orthogonality(q), oracle.residual(x, q, r)
    orth_o, res_o = oracle.orthogonality(q_o), oracle.residual(x, q_o, r_o)
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert orth <= max(10 * orth_o, 1e-13), (orth, orth_o)
    assert res <= max(10 * res_o, 1e-13), (res, res_o)
    if kappa <= 1e6:
        assert np.linalg.norm(r - r_o) / np.linalg.norm(r_o) <= 1e-10 * kappa


@pytest.mark.parametrize("algo", ["rclupp", "rcluppr"])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10, 1e12])
def test_driver_at_reduced_tier(rq, algo, prec, kappa):
    m, n, s = 8192, 64, 128
    x = synth.svd_matrix(m, n, kappa, 71)
    fn = rq.rclupp_factor if algo == "rclupp" else rq.rclupp_r_factor
    Q, R, info = fn(dev(x), s=s, seed=5, prec=prec)
    q_o, r_o, _ = getattr(oracle, algo)(x, S=oracle.gaussian_sketch_matrix(s, m, 5))
    _gate(x, host(Q), host(R), q_o, r_o, kappa)
    assert info.prec_used in (0, 1, 2)
    if kappa <= 1e2:
        assert info.prec_used == prec  # a well-conditioned X needs no escalation
    if algo == "rcluppr" and kappa <= 1e10:
        # RCLUPPr sketches the well-conditioned M: the reduced tier suffices
        assert info.prec_used == prec


def test_escalation_reaches_binary64_when_needed(rq):
    # kappa 1e15: a bf16 sketch leaves Q1 far too ill-conditioned; the driver
    # must escalate and still meet the binary64 result's accuracy
    m, n, s = 8192, 32, 64
    x = synth.svd_matrix(m, n, 1e15, 72)
    Q, R, info = rq.rclupp_factor(dev(x), s=s, seed=6, prec=1, check=False)
    q_o, r_o, st_o = oracle.rclupp(x, S=oracle.gaussian_sketch_matrix(s, m, 6), raise_on_error=False)
    assert info.prec_used != 1
    if st_o == 0 and info.status == 0:
        assert oracle.orthogonality(host(Q)) <= max(1e3 * oracle.orthogonality(q_o), 1e-12)


# ------------------------------------------------------------- digit tier ---

def _digit_tol(z, x, s, m):
    """|Y_gpu - Y_exact| for the digit tier: binary64 roundings of the int64
    flushes and of the ordered sums over windows and CTAs (at most m/1024 + 2
    of them per entry, each 2^-53 of |k| |F|), and level 5's rounding to units
    of 2^8 per 1024-row window (2^(E - 45) each, in units of Y times sqrt(s))."""
    k = np.abs(32 * z)
    E = np.floor(np.log2(np.max(np.abs(x), axis=0) + 1e-300)) + 1
    mag = (k @ (np.abs(x) + 2.0 ** (E - 48))) * 2.0 ** -5
    w = m / 1024 + 2
    return (4 * w * 2.0 ** -53 * mag + w * 2.0 ** (E - 45)) / np.sqrt(s)


@pytest.mark.parametrize("m,n,s", [(1, 1, 1), (100, 7, 8), (4096, 64, 128), (20001, 128, 256),
                                   (3001, 200, 300), (2048, 256, 512), (70000, 33, 66)])
def test_digit_sketch_matches_definition(rq, m, n, s):
    x = synth.svd_matrix(m, n, 1e6, m + n) if m >= n else synth.integer_matrix(m, n, 1)
    seed = 4321 + m
    y = host(rq.rclupp_sketch(dev(x), s=s, seed=seed, prec=rq.PREC_SKETCH_DIGITS))
    ref = oracle.sketch_digits(s, seed, x)
    z = oracle.tier_sketch_z(s, m, seed)
    assert np.all(np.abs(y - ref) <= _digit_tol(z, x, s, m) + 1e-300)


def test_digit_sketch_exact_on_integers_and_scaling(rq):
    # small integers: every digit sum is exact, so the result is the oracle's
    # bit for bit; scaling a column by a power of two scales its sketch exactly
    m, n, s, seed = 5000, 6, 64, 12
    x = synth.integer_matrix(m, n, 4)
    y = host(rq.rclupp_sketch(dev(x), s=s, seed=seed, prec=rq.PREC_SKETCH_DIGITS))
    assert np.array_equal(y, oracle.sketch_digits(s, seed, x))
    sc = 2.0 ** np.array([300, 0, -500, 7, -20, 1000])
    y2 = host(rq.rclupp_sketch(dev(x * sc), s=s, seed=seed, prec=rq.PREC_SKETCH_DIGITS))
    assert np.array_equal(y2, y * sc)


def test_digit_sketch_unit_lower_row_blocks_and_nonfinite(rq):
    m, n, s = 3000, 24, 48
    x = synth.svd_matrix(m, n, 1e4, 8)
    lu, _, _, _ = oracle.gepp(x)
    M = oracle.unit_lower(lu)
    y = host(rq.rclupp_sketch(dev(lu), s=s, seed=4, prec=rq.PREC_SKETCH_DIGITS, unit_lower=True))
    ref = oracle.sketch_digits(s, 4, M)
    assert np.all(np.abs(y - ref) <= _digit_tol(oracle.tier_sketch_z(s, m, 4), M, s, m) + 1e-300)
    # a row block starting at global row row0 draws the global entries
    xi = synth.integer_matrix(301, 5, 2)
    for row0 in (0, 5, 1024):
        yb = host(rq.rclupp_sketch(dev(xi), s=32, seed=9, prec=rq.PREC_SKETCH_DIGITS, row0=row0))
        z = oracle.tier_sketch_z(32, row0 + 301, 9)[:, row0:]
        assert np.array_equal(yb, ((32 * z @ xi) * 2.0 ** -5) * (1.0 / np.sqrt(32))), row0
    # a NaN makes its column NaN, the others are unaffected
    xn = synth.svd_matrix(2000, 4, 10.0, 3)
    xn[77, 2] = np.nan
    yn = host(rq.rclupp_sketch(dev(xn), s=16, seed=1, prec=rq.PREC_SKETCH_DIGITS))
    assert np.all(np.isnan(yn[:, 2])) and np.all(np.isfinite(np.delete(yn, 2, axis=1)))


@pytest.mark.parametrize("algo", ["rclupp", "rcluppr", "rcholqr"])
@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e12, 1e15])
def test_driver_digit_tier_needs_no_escalation(rq, algo, kappa):
    # 48 bits and exact sums leave Q1 well conditioned at any kappa here: the
    # result comes from the digit tier itself, with the binary64 gates
    m, n, s = 8192, 64, 128
    x = synth.svd_matrix(m, n, kappa, 91)
    fn = {"rclupp": rq.rclupp_factor, "rcluppr": rq.rclupp_r_factor, "rcholqr": rq.rcholqr_factor}[algo]
    Q, R, info = fn(dev(x), s=s, seed=8, prec=rq.PREC_SKETCH_DIGITS, check=False)
    assert info.status == 0 and info.prec_used == rq.PREC_SKETCH_DIGITS
    q_o, r_o, st_o = getattr(oracle, algo)(x, S=oracle.gaussian_sketch_matrix(s, m, 8), raise_on_error=False)
    if kappa <= 1e12:
        _gate(x, host(Q), host(R), q_o, r_o, kappa)
    elif algo != "rcholqr":
        assert oracle.orthogonality(host(Q)) <= max(10 * oracle.orthogonality(q_o), 1e-13)
        assert oracle.residual(x, host(Q), host(R)) <= max(10 * oracle.residual(x, q_o, r_o), 1e-13)
