"""Row-sharded RCLUPP and CholeskyQR2 (paper_2412_06551_gb300.distributed).

CPU, gloo, world_size 2 and 3: each rank runs the per-rank steps through the
oracle (plain binary64 C) on its own rows of X, with torch.distributed's
all-reduce between them.  Checked: exactly three all-reduces for RCLUPP (of
s x n, n x n, n x n) and two for CholeskyQR2; every rank ends with the same R;
the stacked Q and R meet the same gates against the single-matrix oracle as
the GPU path (orthogonality and residual within max(10x, 1e-13), R within
1e-10 kappa).  The generated sketch is the whole matrix's: rank r uses the
columns row0 .. row0 + m_r - 1 of the same S.  The GPU form (the library's
steps on one GPU, ranks emulated by summing row blocks in one process) is in
test_gpu_sharded.py.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _rows(A):
    # the library's tall steps take m >= 1 rows (RCLUPP_ERR_ARG otherwise);
    # the scaffolding keeps that contract so a driver cannot rely on less
    if A.shape[0] < 1:
        raise ValueError("tall step called with no rows")
    return A


class OracleSteps:
    """The per-rank steps on the CPU through the oracle (test scaffolding)."""

    def __init__(self, S_full):
        self.S_full = S_full

    def sketch(self, A, *, s, kind, zeta, seed, row0):
        import oracle
        return oracle.sketch_dense(self.S_full[:, row0:row0 + A.shape[0]], _rows(A))

    def precond(self, Y):
        import oracle
        return oracle.sketch_precond(Y)[0]

    def trsm_gram(self, A, R, *, gram):
        import oracle
        Q = oracle.trsm(_rows(A), R)
        return Q, (oracle.gram(Q) if gram else None)

    def gram(self, A):
        import oracle
        return oracle.gram(_rows(A))

    def cholesky(self, G):
        import oracle
        return oracle.cholesky(G, raise_on_error=False)

    def trmm(self, A, B):
        import oracle
        return oracle.trmm_upper(A, B)

    def zeros(self, like, rows, cols):
        return np.zeros((rows, cols), order="F")


def _problem(m, n, kappa):
    import synth
    import oracle
    x = synth.svd_matrix(m, n, kappa, 4242)
    S = oracle.gaussian_sketch_matrix(2 * n, m, 77)
    return x, S


def _worker(rank, world, port, algo, m, n, kappa, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2412_06551_gb300 import distributed as D
    x, S = _problem(m, n, kappa)
    row0, rows = D.row_block(m, world, rank)
    sizes = []

    def allreduce(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        sizes.append(tuple(a.shape))
        return np.asfortranarray(t.numpy())

    steps = OracleSteps(S)
    xl = np.asfortranarray(x[row0:row0 + rows])
    if algo == "rclupp":
        Q, R = D.rclupp_factor_sharded(xl, row0, s=2 * n, seed=77, steps=steps, allreduce=allreduce)
    else:
        Q, R = D.cholqr2_factor_sharded(xl, steps=steps, allreduce=allreduce)
    q.put((rank, row0, Q, R, sizes))
    dist.destroy_process_group()


def _run(world, port, algo, m, n, kappa):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, algo, m, n, kappa, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda t: t[0])


@pytest.mark.parametrize("world,port", [(2, 29561), (3, 29562)])
@pytest.mark.parametrize("kappa", [1e4, 1e12])
def test_rclupp_sharded_matches_single_matrix_oracle(world, port, kappa):
    import oracle
    m, n = 3001, 24
    out = _run(world, port + (0 if kappa < 1e6 else 10), "rclupp", m, n, kappa)
    x, S = _problem(m, n, kappa)
    Q = np.vstack([o[2] for o in out])
    R = out[0][3]
    for o in out:
        assert np.array_equal(o[3], R)                       # the same R everywhere
        assert o[4] == [(2 * n, n), (n, n), (n, n)]           # three all-reduces
    q_o, r_o, _ = oracle.rclupp(x, S=S)
    orth, res = oracle.orthogonality(Q), oracle.residual(x, Q, R)
    assert orth <= max(10 * oracle.orthogonality(q_o), 1e-13)
    assert res <= max(10 * oracle.residual(x, q_o, r_o), 1e-13)
    if kappa <= 1e6:
        assert np.linalg.norm(R - r_o) / np.linalg.norm(r_o) <= 1e-10 * kappa


def test_cholqr2_sharded_two_allreduces():
    import oracle
    m, n = 2000, 16
    out = _run(2, 29581, "cholqr2", m, n, 1e3)
    x, _ = _problem(m, n, 1e3)
    Q = np.vstack([o[2] for o in out])
    R = out[0][3]
    assert all(o[4] == [(n, n), (n, n)] for o in out)
    q_o, r_o, _ = oracle.cholqr2(x)
    assert oracle.orthogonality(Q) <= max(10 * oracle.orthogonality(q_o), 1e-13)
    assert np.linalg.norm(R - r_o) / np.linalg.norm(r_o) <= 1e-10 * 1e3


@pytest.mark.parametrize("algo,port", [("rclupp", 29565), ("cholqr2", 29566)])
def test_rank_without_rows_still_joins_every_allreduce(algo, port):
    # three ranks, two rows: rank 2 holds none and adds zero partials; all
    # ranks make the same all-reduces and end with the same R
    import oracle
    world, m, n = 3, 2, 2
    out = _run(world, port, algo, m, n, 1e3)
    assert [o[2].shape[0] for o in out] == [1, 1, 0]
    x, S = _problem(m, n, 1e3)
    Q = np.vstack([o[2] for o in out])
    R = out[0][3]
    expect = [(2 * n, n), (n, n), (n, n)] if algo == "rclupp" else [(n, n), (n, n)]
    for o in out:
        assert np.array_equal(o[3], R)
        assert o[4] == expect
    q_o, r_o, _ = oracle.rclupp(x, S=S) if algo == "rclupp" else oracle.cholqr2(x)
    assert oracle.orthogonality(Q) <= max(10 * oracle.orthogonality(q_o), 1e-13)
    assert oracle.residual(x, Q, R) <= max(10 * oracle.residual(x, q_o, r_o), 1e-13)
    assert np.linalg.norm(R - r_o) / np.linalg.norm(r_o) <= 1e-10 * 1e3


def test_torch_allreduce_passes_contiguous_tensors_and_sums_in_place(monkeypatch):
    # NCCL rejects non-contiguous tensors; the library's matrices are
    # column-major views.  A stand-in all_reduce that insists on contiguous
    # input and doubles it (two ranks holding the same values) checks that
    # every layout is reduced in place with the right result.
    from paper_2412_06551_gb300 import distributed as D
    seen = []

    def fake_all_reduce(t, op=None, group=None):
        assert t.is_contiguous()
        seen.append(tuple(t.shape))
        t.mul_(2)

    monkeypatch.setattr(dist, "all_reduce", fake_all_reduce)
    reduce_ = D.torch_allreduce()
    base = torch.arange(12, dtype=torch.float64)
    col = base.clone().reshape(3, 4).t()                   # 4 x 3 column-major (ld = 4)
    row = base.clone().reshape(4, 3)                       # row-major
    padded = base.clone().reshape(3, 4).t()[:3]            # 3 x 3 column-major, ld = 4
    for t in (col, row, padded):
        before = t.clone()
        ptr = t.data_ptr()
        out = reduce_(t)
        assert out is t and t.data_ptr() == ptr
        assert torch.equal(t, 2 * before)
    assert seen == [(3, 4), (4, 3), (3, 3)]


def test_srht_needs_the_whole_matrix_order():
    from paper_2412_06551_gb300 import distributed as D
    import paper_2412_06551_gb300 as rq
    with pytest.raises(ValueError):
        D.rclupp_factor_sharded(np.zeros((10, 2)), 0, kind=rq.SKETCH_SRHT, steps=OracleSteps(None),
                                allreduce=lambda a: a)


def test_row_block_partition():
    from paper_2412_06551_gb300.distributed import row_block
    for m in (1, 7, 100, 3001):
        for world in (1, 2, 3, 8):
            blocks = [row_block(m, world, r) for r in range(world)]
            assert blocks[0][0] == 0
            assert sum(b[1] for b in blocks) == m
            for (a0, an), (b0, _) in zip(blocks, blocks[1:]):
                assert a0 + an == b0


def _failing_worker(rank, world, port, algo, q):
    # a numerical failure is decided on replicated, all-reduced data, so every
    # rank raises at the same point and none is left waiting in a collective
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2412_06551_gb300 import distributed as D
    m, n = 3000, 24
    x, S = _problem(m, n, 1e12 if algo == "cholqr2" else 1e4)
    if algo == "rclupp":
        x[:, 7] = 0.0  # the sketch has a zero column: zero pivot in its LU
    row0, rows = D.row_block(m, world, rank)
    sizes = []

    def allreduce(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        sizes.append(tuple(a.shape))
        return np.asfortranarray(t.numpy())

    xl = np.asfortranarray(x[row0:row0 + rows])
    try:
        if algo == "rclupp":
            D.rclupp_factor_sharded(xl, row0, s=2 * n, seed=77, steps=OracleSteps(S), allreduce=allreduce)
        else:
            D.cholqr2_factor_sharded(xl, steps=OracleSteps(S), allreduce=allreduce)
        q.put((rank, "ok", None, None, sizes))
    except oracle.OracleError as e:
        q.put((rank, "oracle", e.status, e.info, sizes))
    except Exception as e:  # the library's error type
        q.put((rank, type(e).__name__, getattr(e, "status", None), getattr(e, "column", None), sizes))
    dist.barrier()  # every rank is past the failure: nobody waits in a collective
    dist.destroy_process_group()


@pytest.mark.parametrize("algo,port", [("cholqr2", 29563), ("rclupp", 29564)])
def test_sharded_failure_is_raised_on_every_rank(algo, port):
    import oracle
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_failing_worker, args=(r, world, port, algo, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=240) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    kinds = {o[1:4] for o in out}
    assert len(kinds) == 1, out  # the same failure, status and column on every rank
    kind, status, col = kinds.pop()
    if algo == "cholqr2":
        assert kind == "RclupError" and status == oracle.CHOL_BREAKDOWN and col >= 1
        assert all(o[4] == [(24, 24)] for o in out)  # failed in the first pass, after one all-reduce
    else:
        # the replicated preconditioner's LU (through the oracle here) finds the zero pivot
        assert kind == "oracle" and status == oracle.LU_ZERO_PIVOT and col == 7
        assert all(o[4] == [(48, 24)] for o in out)  # only the sketch was all-reduced
