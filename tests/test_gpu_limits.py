"""The largest supported sizes and the boundaries between kernel forms, on
the GPU through the C ABI, against the oracle.

* Sketch size s: up to 4096 for the Gaussian sketch (binary64 and the
  tensor-core tiers) and the drivers; up to 768 for the sparse-sign sketch,
  whose accumulators for all s rows live in shared memory; beyond them the
  call returns RCLUPP_ERR_UNSUPPORTED before any launch.
* The preconditioner of Algorithms 5-7 (small LU, R-factor of
  HouseholderQR, R1 = R0 N) runs in one thread block cluster while the s x n
  matrix fits the cluster's shared memory (at most 8 CTAs of 200 KB: s <= 776
  at n = 256, s <= 1576 at n = 128) and in one CTA working in global memory
  beyond that; both sides of each boundary are compared with the oracle.
* A square X (m = n = 256), the smallest tall-skinny shape.
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


def gamma32(k):
    u = 2.0 ** -24
    return k * u / (1 - k * u)


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


def _gate(x, q, r, q_o, r_o, kappa):
    orth, res = oracle.orthogonality(q), oracle.residual(x, q, r)
    orth_o, res_o = oracle.orthogonality(q_o), oracle.residual(x, q_o, r_o)
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
    assert orth <= max(10 * orth_o, 1e-13), (orth, orth_o)
    assert res <= max(10 * res_o, 1e-13), (res, res_o)
    if kappa <= 1e6:
        assert np.linalg.norm(r - r_o) / np.linalg.norm(r_o) <= 1e-10 * kappa


# ------------------------------------------------------------ sketch sizes ---

def test_gaussian_sketch_at_the_largest_s(rq):
    m, n, s, seed = 3001, 65, 4096, 2 ** 33 + 17
    x = synth.svd_matrix(m, n, 1e2, 8)
    y = host(rq.rclupp_sketch(dev(x), s=s, seed=seed))
    S = oracle.gaussian_sketch_matrix(s, m, seed)
    ref = oracle.sketch_dense(S, x)
    assert np.all(np.abs(y - ref) <= 2 * gamma(m) * (np.abs(S) @ np.abs(x)) + 1e-300)


@pytest.mark.parametrize("prec,nterms", [(1, 1), (2, 3)])
def test_tensor_core_sketch_at_the_largest_s(rq, prec, nterms):
    m, n, s, seed = 3001, 65, 4096, 99
    x = synth.svd_matrix(m, n, 1e2, 9)
    y = host(rq.rclupp_sketch(dev(x), s=s, seed=seed, prec=prec))
    ref = oracle.sketch_bf16(s, seed, nterms, x)
    S = oracle.tier_sketch_z(s, m, seed) / np.sqrt(s)
    mag = (1 + 2.0 ** -7) * (np.abs(S) @ np.abs(x))
    assert np.all(np.abs(y - ref) <= gamma32(m) * mag + 1e-300)


def test_sparse_sign_sketch_at_the_largest_s(rq):
    m, n, s, zeta, seed = 3001, 40, 768, 8, 21
    x = synth.svd_matrix(m, n, 1e2, 10)
    y = host(rq.rclupp_sketch(dev(x), s=s, kind=rq.SKETCH_SPARSE_SIGN, zeta=zeta, seed=seed))
    rows, signs = oracle.sparse_sign_pattern(s, m, zeta, seed)
    ref = oracle.sketch_sparse(s, zeta, rows, signs, x)
    S = oracle.sparse_to_dense(s, m, zeta, rows, signs)
    assert np.all(np.abs(y - ref) <= 2 * gamma(m) * (np.abs(S) @ np.abs(x)) + 1e-300)


def test_sizes_beyond_the_limits_are_unsupported(rq):
    x = dev(synth.svd_matrix(5000, 40, 10.0, 11))
    cases = [lambda: rq.rclupp_sketch(x, s=769, kind=rq.SKETCH_SPARSE_SIGN, zeta=8),
             lambda: rq.rclupp_sketch(x, s=4097),
             lambda: rq.rclupp_factor(x, s=4097),
             lambda: rq.rclupp_r_factor(x, s=4097),
             lambda: rq.rcholqr_factor(x, s=4097)]
    for call in cases:
        with pytest.raises(rq.RclupError) as e:
            call()
        assert e.value.status == rq.Status.ERR_UNSUPPORTED


# ----------------------------------------- preconditioner: cluster / one CTA ---

@pytest.mark.parametrize("s,n,kappa", [(776, 256, 1e4), (777, 256, 1e4), (1576, 128, 1e6),
                                       (1577, 128, 1e6), (4096, 256, 1e2), (4096, 16, 1e8)])
def test_sketch_precond_on_both_sides_of_the_cluster_limit(rq, s, n, kappa):
    y = synth.svd_matrix(s, n, kappa, s + n)
    r1 = host(rq.rclupp_sketch_precond(dev(y)))
    r1_ref, _, _ = oracle.sketch_precond(y)
    assert np.all(np.diag(r1) > 0) and np.array_equal(r1, np.triu(r1))
    assert np.linalg.norm(r1 - r1_ref) <= 1000 * n * U * kappa * np.linalg.norm(r1_ref)


@pytest.mark.parametrize("algo", ["rclupp", "rcluppr", "rcholqr"])
@pytest.mark.parametrize("m,n,s,kappa", [(5000, 128, 4096, 1e6), (3000, 256, 1024, 1e4)])
def test_drivers_with_the_one_cta_preconditioner(rq, algo, m, n, s, kappa):
    x = synth.svd_matrix(m, n, kappa, m + s)
    fn = {"rclupp": rq.rclupp_factor, "rcluppr": rq.rclupp_r_factor, "rcholqr": rq.rcholqr_factor}[algo]
    Q, R, _ = fn(dev(x), s=s, seed=12)
    q_o, r_o, _ = getattr(oracle, algo)(x, S=oracle.gaussian_sketch_matrix(s, m, 12))
    _gate(x, host(Q), host(R), q_o, r_o, kappa)


# ------------------------------------------------------------- square X ---

@pytest.mark.parametrize("algo", ["rclupp", "rcluppr", "cholqr2", "lc2", "rcholqr", "scholqr3"])
def test_square_x(rq, algo):
    n, kappa = 256, 1e2
    x = synth.svd_matrix(n, n, kappa, 13)
    X = dev(x)
    if algo in ("rclupp", "rcluppr", "rcholqr"):
        fn = {"rclupp": rq.rclupp_factor, "rcluppr": rq.rclupp_r_factor, "rcholqr": rq.rcholqr_factor}[algo]
        Q, R, _ = fn(X, s=2 * n, seed=14)
        q_o, r_o, _ = getattr(oracle, algo)(x, S=oracle.gaussian_sketch_matrix(2 * n, n, 14))
    else:
        fn = {"cholqr2": rq.cholqr2_factor, "lc2": rq.lc2_factor, "scholqr3": rq.scholqr3_factor}[algo]
        Q, R, _ = fn(X)
        q_o, r_o, _ = getattr(oracle, algo)(x)
    _gate(x, host(Q), host(R), q_o, r_o, kappa)
