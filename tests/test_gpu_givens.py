"""Parity of the Givens-rotation R-factor (the alternative R0 of Section 1 and
of the remark after Algorithm 5) with the oracle, through the C ABI.

The device kernel rotates each column's subcolumn away by a tree (within each
CTA's rows, then across the CTAs' head rows), the oracle bottom-up row by
row: both give the unique R with a non-negative diagonal, so they agree to
the forward error of a backward-stable QR, O(s u kappa(A)) relative.  Inputs
that need no rotation (already upper triangular) are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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


def _pos(r):
    return np.sign(np.where(np.diag(r) == 0, 1.0, np.diag(r)))[:, None] * r


@pytest.mark.parametrize("s,n", [(2, 1), (17, 5), (64, 32), (100, 100), (256, 128), (300, 150),
                                 (512, 256), (1000, 16), (3000, 8)])
def test_givens_r_matches_oracle(rq, s, n):
    a = np.random.default_rng(s + n).standard_normal((s, n))
    r = host(rq.rclupp_givens_r(dev(a)))
    r_ref = _pos(oracle.givens_r(a))
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) >= 0)
    assert np.linalg.norm(r - r_ref) <= 100 * s * U * np.linalg.cond(a) * np.linalg.norm(r_ref)


def test_givens_r_needs_no_rotation_on_upper_input(rq):
    u = np.triu(np.random.default_rng(4).standard_normal((300, 40)))
    u[:40][np.diag_indices(40)] = np.abs(np.diag(u[:40])) + 1.0
    assert np.array_equal(host(rq.rclupp_givens_r(dev(u))), u[:40])


def test_givens_r_one_column_is_the_norm(rq):
    a = np.random.default_rng(5).standard_normal((2000, 1))
    r = host(rq.rclupp_givens_r(dev(a)))[0, 0]
    assert abs(r - np.linalg.norm(a)) <= 16 * U * np.linalg.norm(a)
    assert host(rq.rclupp_givens_r(dev(np.array([[3.0], [4.0]]))))[0, 0] == 5.0


@pytest.mark.parametrize("s,n,kappa", [(4, 2, 10.0), (64, 32, 1e4), (256, 128, 1e8), (300, 150, 1e2),
                                       (512, 256, 1e6)])
def test_sketch_precond_givens(rq, s, n, kappa):
    y = synth.svd_matrix(s, n, kappa, s)
    r1 = host(rq.rclupp_sketch_precond(dev(y), r0=rq.R0_GIVENS))
    r1_ref, _, _ = oracle.sketch_precond(y, r0="givens")
    assert np.all(np.diag(r1) > 0) and np.array_equal(r1, np.triu(r1))
    assert np.linalg.norm(r1 - r1_ref) <= 1000 * n * U * kappa * np.linalg.norm(r1_ref)


def _gate(x, q, r, q_o, r_o, kappa):
    orth, res = oracle.orthogonality(q), oracle.residual(x, q, r)
    orth_o, res_o = oracle.orthogonality(q_o), oracle.residual(x, q_o, r_o)
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert orth <= max(10 * orth_o, 1e-13), (orth, orth_o)
    assert res <= max(10 * res_o, 1e-13), (res, res_o)
    if kappa <= 1e6:
        assert np.linalg.norm(r - r_o) / np.linalg.norm(r_o) <= 1e-10 * kappa


@pytest.mark.parametrize("algo", ["rclupp", "rcluppr", "rcholqr"])
@pytest.mark.parametrize("kappa", [1e4, 1e12])
def test_drivers_with_givens_r0(rq, algo, kappa):
    m, n, s = 8000, 64, 128
    if algo == "rcholqr":
        kappa = min(kappa, 1e6)  # one CholeskyQR after the sketch (Algorithm 5)
    x = synth.svd_matrix(m, n, kappa, 47)
    fn = {"rclupp": rq.rclupp_factor, "rcluppr": rq.rclupp_r_factor, "rcholqr": rq.rcholqr_factor}[algo]
    Q, R, _ = fn(dev(x), s=s, seed=3, r0=rq.R0_GIVENS)
    S = oracle.gaussian_sketch_matrix(s, m, 3)
    q_o, r_o, _ = getattr(oracle, algo)(x, S=S, r0="givens")
    _gate(x, host(Q), host(R), q_o, r_o, kappa)


def test_givens_batched_matches_single_calls(rq):
    g = np.random.default_rng(8)
    xs = [synth.svd_matrix(int(mm), int(nn), 1e6, 950 + i)
          for i, (mm, nn) in enumerate(zip(g.integers(300, 5000, 8), g.choice([8, 33, 64, 100], 8)))]
    Xs = [dev(x) for x in xs]
    for algo, fn in [(rq.ALGO_RCLUPP, rq.rclupp_factor), (rq.ALGO_RCLUPPR, rq.rclupp_r_factor)]:
        Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=algo, seed=31, r0=rq.R0_GIVENS)
        assert np.all(st == 0)
        for i, X in enumerate(Xs):
            q, r, _ = fn(X, s=2 * X.shape[1], seed=31 + i, r0=rq.R0_GIVENS)
            assert torch.equal(Qb[i], q) and torch.equal(Rb[i], r), (algo, i)


def test_givens_unsupported_beyond_a_cluster(rq):
    x = dev(synth.svd_matrix(8192, 256, 10.0, 1))
    with pytest.raises(rq.RclupError) as e:  # s x n = 4096 x 256 does not fit 8 CTAs
        rq.rclupp_factor(x, s=4096, r0=rq.R0_GIVENS)
    assert e.value.status == rq.Status.ERR_UNSUPPORTED
    with pytest.raises(rq.RclupError):
        rq.rclupp_factor(x, s=512, r0=7)


@pytest.mark.slow
def test_givens_full_size_m1M_n128(rq):
    m, n, s = 1 << 20, 128, 256
    x = synth.svd_matrix(m, n, 1e4, synth.kappa_seed(1, 0))
    X = dev(x)
    Q, R, _ = rq.rclupp_factor(X, s=s, seed=7, r0=rq.R0_GIVENS)
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert float(torch.linalg.norm(Q.t() @ Q - eye)) <= 1e-13
    assert float(torch.linalg.norm(Q @ R - X) / torch.linalg.norm(X)) <= 1e-13
    _, Rh, _ = rq.rclupp_factor(X, s=s, seed=7)
    r, rh = host(R), host(Rh)
    assert np.linalg.norm(r - rh) / np.linalg.norm(rh) <= 1e-10 * 1e4
