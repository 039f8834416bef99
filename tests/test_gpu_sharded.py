"""The GPU pieces of the row-sharded driver (paper_2412_06551_gb300.distributed).

The multi-rank structure runs on CPU ranks in test_sharded.py (one GPU per
run here, and ranks whose collectives wait on one another must not share a
GPU).  On the GPU: the sketch of a row block (rclupp_sketch_rows) is the
corresponding partial of the whole matrix's generated sketch, and the
driver with one rank (the all-reduce an identity) gives the single-call
factorization bit for bit, since it runs the same kernels in the same order.
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
    a = np.asfortranarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda").t()


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


@pytest.fixture(scope="module")
def rq():
    import paper_2412_06551_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("m,n,world", [(5000, 32, 2), (7001, 100, 3), (4096, 256, 4)])
def test_row_block_sketch_is_the_partial_of_the_full_sketch(rq, kind, m, n, world):
    from paper_2412_06551_gb300.distributed import row_block
    x = synth.svd_matrix(m, n, 1e3, m + n)
    s, seed = 2 * n, 99
    parts = []
    for r in range(world):
        row0, rows = row_block(m, world, r)
        parts.append(host(rq.rclupp_sketch(dev(x[row0:row0 + rows]), s=s, kind=kind, zeta=4,
                                           seed=seed, row0=row0)))
        if kind == 0:  # each partial against the oracle's slice of the same S
            S = oracle.gaussian_sketch_matrix(s, m, seed)[:, row0:row0 + rows]
            ref = oracle.sketch_dense(S, x[row0:row0 + rows])
            bound = 2 * gamma(rows) * (np.abs(S) @ np.abs(x[row0:row0 + rows]))
            assert np.all(np.abs(parts[-1] - ref) <= bound + 1e-300)
    full = host(rq.rclupp_sketch(dev(x), s=s, kind=kind, zeta=4, seed=seed))
    total = sum(parts)
    if kind == 0:
        S = oracle.gaussian_sketch_matrix(s, m, seed)
        bound = 3 * gamma(m) * (np.abs(S) @ np.abs(x))
    else:
        rows_, signs = oracle.sparse_sign_pattern(s, m, 4, seed)
        bound = 3 * gamma(m) * oracle.sketch_sparse(s, 4, rows_, np.ones_like(signs), np.abs(x))
    assert np.all(np.abs(total - full) <= bound + 1e-300)


@pytest.mark.parametrize("m,n,kappa", [(20000, 64, 1e6), (9000, 128, 1e10)])
def test_single_rank_driver_equals_single_call(rq, m, n, kappa):
    from paper_2412_06551_gb300 import distributed as D
    x = synth.svd_matrix(m, n, kappa, 5 * n)
    X = dev(x)
    ident = lambda t: t
    Q, R = D.rclupp_factor_sharded(X, 0, s=2 * n, seed=13, allreduce=ident)
    Q1, R1, _ = rq.rclupp_factor(X, s=2 * n, seed=13)
    assert torch.equal(R, R1) and torch.equal(Q, Q1)
    Qc, Rc = D.cholqr2_factor_sharded(X, allreduce=ident) if kappa < 1e7 else (None, None)
    if Qc is not None:
        Qc1, Rc1, _ = rq.cholqr2_factor(X)
        assert oracle.orthogonality(host(Qc)) <= max(10 * oracle.orthogonality(host(Qc1)), 1e-13)
        assert np.linalg.norm(host(Rc) - host(Rc1)) <= 1e-12 * np.linalg.norm(host(Rc1))


def test_two_blocks_summed_on_one_gpu(rq):
    # two "ranks" run step by step in one process, their partials summed on
    # the GPU: the result meets the single-matrix oracle's gates
    from paper_2412_06551_gb300.distributed import LibrarySteps, row_block
    m, n, kappa = 12000, 48, 1e8
    x = synth.svd_matrix(m, n, kappa, 31)
    steps = LibrarySteps()
    blocks = [row_block(m, 2, r) for r in range(2)]
    Xs = [dev(x[r0:r0 + rows]) for r0, rows in blocks]
    Y = sum(steps.sketch(Xb, s=2 * n, kind=0, zeta=8, seed=5, row0=r0) for Xb, (r0, _) in zip(Xs, blocks))
    R1 = steps.precond(Y)
    QG = [steps.trsm_gram(Xb, R1, gram=True) for Xb in Xs]
    R2, st, _ = steps.cholesky(sum(g for _, g in QG))
    assert st == 0
    QG2 = [steps.trsm_gram(q, R2, gram=True) for q, _ in QG]
    R4, st, _ = steps.cholesky(sum(g for _, g in QG2))
    assert st == 0
    Q = torch.cat([steps.trsm_gram(q, R4, gram=False)[0] for q, _ in QG2], dim=0)
    R = steps.trmm(R4, steps.trmm(R2, R1))
    q_o, r_o, _ = oracle.rclupp(x, S=oracle.gaussian_sketch_matrix(2 * n, m, 5))
    q, r = host(Q), host(R)
    assert oracle.orthogonality(q) <= max(10 * oracle.orthogonality(q_o), 1e-13)
    assert oracle.residual(x, q, r) <= max(10 * oracle.residual(x, q_o, r_o), 1e-13)


def test_single_rank_driver_srht_equals_single_call(rq):
    import oracle as orc
    from paper_2412_06551_gb300 import distributed as D
    m, n = 7000, 40
    x = synth.svd_matrix(m, n, 1e6, 77)
    X = dev(x)
    b = orc.srht_order_log2(m)
    Q, R = D.rclupp_factor_sharded(X, 0, s=2 * n, seed=13, kind=rq.SKETCH_SRHT, order_log2=b,
                                   allreduce=lambda t: t)
    Q1, R1, _ = rq.rclupp_factor(X, s=2 * n, seed=13, kind=rq.SKETCH_SRHT)
    assert torch.equal(R, R1) and torch.equal(Q, Q1)
