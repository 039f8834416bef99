"""Batched form: many uneven factorizations in one graph launch.

The batch runs the same kernels as single calls with the same launch
shapes, so every problem's Q and R must equal the single call's bit for bit;
against the oracle they meet the usual gates.  Each problem reports its own
status.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _batch(count, seed, nmax=128):
    g = np.random.default_rng(seed)
    ns = g.choice([1, 3, 16, 33, 64, 96, nmax], size=count)
    ms = np.maximum(ns, np.exp(g.uniform(np.log(64), np.log(6000), size=count)).astype(int))
    kap = 10.0 ** g.uniform(1, 8, size=count)
    xs = [synth.svd_matrix(int(m), int(n), float(k), 1000 + i) for i, (m, n, k) in enumerate(zip(ms, ns, kap))]
    return xs, kap


ALGOS = [(0, "rclupp"), (1, "rcluppr"), (2, "cholqr2"), (3, "lc2")]


@pytest.mark.parametrize("algo,name", ALGOS)
def test_batched_equals_single_calls(rq, algo, name):
    xs, kap = _batch(20, algo + 5)
    Xs = [dev(x) for x in xs]
    Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=algo, seed=77)
    assert np.all(st == 0)
    for i, X in enumerate(Xs):
        if algo == 0:
            Q, R, _ = rq.rclupp_factor(X, seed=77 + i)
        elif algo == 1:
            Q, R, _ = rq.rclupp_r_factor(X, seed=77 + i)
        elif algo == 2:
            Q, R, _ = rq.cholqr2_factor(X)
        else:
            Q, R, _ = rq.lc2_factor(X)
        assert torch.equal(Q, Qb[i]) and torch.equal(R, Rb[i]), i


@pytest.mark.parametrize("algo,name", ALGOS)
def test_batched_against_oracle(rq, algo, name):
    xs, kap = _batch(8, algo + 50, nmax=64)
    Xs = [dev(x) for x in xs]
    Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=algo, seed=5)
    for i, x in enumerate(xs):
        m, n = x.shape
        if name == "rclupp":
            q_o, r_o, _ = oracle.rclupp(x, S=oracle.gaussian_sketch_matrix(2 * n, m, 5 + i))
        elif name == "rcluppr":
            q_o, r_o, _ = oracle.rcluppr(x, S=oracle.gaussian_sketch_matrix(2 * n, m, 5 + i))
        else:
            q_o, r_o, _ = getattr(oracle, name)(x)
        q, r = host(Qb[i]), host(Rb[i])
        assert oracle.orthogonality(q) <= max(10 * oracle.orthogonality(q_o), 1e-13)
        assert oracle.residual(x, q, r) <= max(10 * oracle.residual(x, q_o, r_o), 1e-13)
        if kap[i] <= 1e6:
            assert np.linalg.norm(r - r_o) / np.linalg.norm(r_o) <= 1e-10 * kap[i]


def test_graph_is_reused_and_rebuilt(rq):
    xs, _ = _batch(10, 9)
    Xs = [dev(x) for x in xs]
    Q1, R1, _ = rq.rclupp_factor_batched(Xs, seed=3)
    Q2, R2, _ = rq.rclupp_factor_batched(Xs, Qs=Q1 and None, seed=3)  # new outputs: new graph
    for a, b in zip(R1, R2):
        assert torch.equal(a, b)
    Q3, R3, _ = rq.rclupp_factor_batched(Xs, Qs=Q2, Rs=R2, seed=3)   # same pointers: cached graph
    for a, b in zip(R1, R3):
        assert torch.equal(a, b)
    rq.rclupp_set_batch_branches(3)
    Q4, R4, _ = rq.rclupp_factor_batched(Xs, seed=3)                  # other branch count
    for a, b in zip(R1, R4):
        assert torch.equal(a, b)
    rq.rclupp_set_batch_branches(16)


def test_per_problem_status(rq):
    good = synth.svd_matrix(500, 8, 1e2, 1)
    bad = np.zeros((400, 8))
    bad[:, 0] = 1.0  # rank 1: Cholesky breaks down
    Qb, Rb, st = rq.rclupp_factor_batched([dev(good), dev(bad), dev(good)], algo=2, check=False)
    assert st[0] == 0 and st[2] == 0
    assert st[1] == rq.Status.ERR_CHOL_BREAKDOWN


@pytest.mark.parametrize("prec", [3, 4])
def test_batched_emulated_matches_single_calls(rq, prec):
    # the batched form keeps a binary64 sketch; with the sparse-sign sketch
    # (binary64 at every tier) each problem must equal the single call with
    # the same emulated products bit for bit
    g = np.random.default_rng(prec)
    xs = [synth.svd_matrix(int(m), int(n), 1e6, 700 + i)
          for i, (m, n) in enumerate(zip(g.integers(300, 6000, 10), g.choice([8, 33, 64, 100, 128], 10)))]
    Xs = [dev(x) for x in xs]
    fns = {rq.ALGO_RCLUPP: rq.rclupp_factor, rq.ALGO_RCLUPPR: rq.rclupp_r_factor,
           rq.ALGO_RCHOLQR: rq.rcholqr_factor}
    for algo, fn in fns.items():
        Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=algo, seed=31, prec=prec,
                                              kind=rq.SKETCH_SPARSE_SIGN, zeta=4)
        assert np.all(st == 0)
        for i, X in enumerate(Xs):
            n = X.shape[1]
            q, r, info = fn(X, s=2 * n, seed=31 + i, prec=prec, kind=rq.SKETCH_SPARSE_SIGN, zeta=4)
            assert torch.equal(Qb[i], q) and torch.equal(Rb[i], r), (algo, i)
            assert info.emulated == prec - 2


@pytest.mark.parametrize("prec", [3, 4])
def test_batched_emulated_gaussian_gates(rq, prec):
    g = np.random.default_rng(10 + prec)
    xs = [synth.svd_matrix(int(m), int(n), 10.0 ** g.uniform(2, 10), 800 + i)
          for i, (m, n) in enumerate(zip(g.integers(300, 6000, 12), g.choice([16, 48, 96, 128], 12)))]
    Xs = [dev(x) for x in xs]
    Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=rq.ALGO_RCLUPP, seed=41, prec=prec)
    assert np.all(st == 0)
    for i, x in enumerate(xs):
        m, n = x.shape
        q_o, r_o, _ = oracle.rclupp(x, S=oracle.gaussian_sketch_matrix(2 * n, m, 41 + i))
        q, r = host(Qb[i]), host(Rb[i])
        assert oracle.orthogonality(q) <= max(10 * oracle.orthogonality(q_o), 1e-13)
        assert oracle.residual(x, q, r) <= max(10 * oracle.residual(x, q_o, r_o), 1e-13)


@pytest.mark.parametrize("grid_div,fine", [(4, True), (2, False), (8, True)])
def test_batch_policy_changes_only_the_sum_order(rq, grid_div, fine):
    # smaller launches or row tiles inside the graph: the same factorizations
    # up to the order of the split-K sums, replayed bit for bit
    xs, kap = _batch(16, 40 + grid_div)
    Xs = [dev(x) for x in xs]
    Qd, Rd, st = rq.rclupp_factor_batched(Xs, algo=0, seed=5)
    assert np.all(st == 0)
    try:
        rq.rclupp_set_batch_policy(grid_div, fine)
        assert rq.rclupp_get_batch_policy()[1:] == (grid_div, int(fine))
        Qp, Rp, st2 = rq.rclupp_factor_batched(Xs, algo=0, seed=5)
        first = [(q.clone(), r.clone()) for q, r in zip(Qp, Rp)]
        rq.rclupp_factor_batched(Xs, algo=0, seed=5, Qs=Qp, Rs=Rp)  # cached graph, replayed
    finally:
        rq.rclupp_set_batch_policy(1, False)
    assert np.all(st2 == 0)
    for i, x in enumerate(xs):
        assert torch.equal(Qp[i], first[i][0]) and torch.equal(Rp[i], first[i][1]), i
        q, r, qd, rd = host(Qp[i]), host(Rp[i]), host(Qd[i]), host(Rd[i])
        assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)
        assert oracle.orthogonality(q) <= max(10 * oracle.orthogonality(qd), 1e-13), i
        assert oracle.residual(x, q, r) <= max(10 * oracle.residual(x, qd, rd), 1e-13), i


def test_autotuner_sets_a_valid_policy(rq):
    xs, _ = _batch(12, 91)
    Xs = [dev(x) for x in xs]
    try:
        branches, ms = rq.rclupp_autotune_batched(Xs, algo=0, seed=3)
        b, g, f = rq.rclupp_get_batch_policy()
        assert b == branches and b in (4, 8, 16) and g in (1, 2, 4, 8) and f in (0, 1) and ms > 0
        Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=0, seed=3)
        assert np.all(st == 0)
        for i, x in enumerate(xs):
            assert oracle.orthogonality(host(Qb[i])) <= 1e-13
    finally:
        rq.rclupp_set_batch_branches(16)
        rq.rclupp_set_batch_policy(1, False)


def test_batched_three_term_sketch_matches_single_calls(rq):
    # a batch cannot escalate, so RCLUPP_PREC_SKETCH_FP32 runs the three-term
    # tensor-core sketch for every problem; on inputs where the single call
    # keeps that tier (no escalation) the two are the same kernels with the
    # same launch shapes, bit for bit
    g = np.random.default_rng(17)
    xs = [synth.svd_matrix(int(m), int(n), 1e5, 900 + i)
          for i, (m, n) in enumerate(zip(g.integers(300, 6000, 10), g.choice([8, 33, 64, 100, 128], 10)))]
    Xs = [dev(x) for x in xs]
    Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=rq.ALGO_RCLUPP, seed=61, prec=rq.PREC_SKETCH_FP32)
    assert np.all(st == 0)
    for i, X in enumerate(Xs):
        q, r, info = rq.rclupp_factor(X, seed=61 + i, prec=rq.PREC_SKETCH_FP32)
        assert info.prec_used == rq.PREC_SKETCH_FP32
        assert torch.equal(Qb[i], q) and torch.equal(Rb[i], r), i


def test_batched_bf16_sketch_is_refused(rq):
    # the bf16 tier depends on escalation, which a graph cannot make
    Xs = [dev(synth.svd_matrix(500, 8, 1e2, 1))]
    with pytest.raises(rq.RclupError) as e:
        rq.rclupp_factor_batched(Xs, algo=rq.ALGO_RCLUPP, prec=rq.PREC_SKETCH_BF16)
    assert e.value.status == rq.Status.ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", [2, 3, 4, 5])
def test_batched_tensor_core_sketch_gates_up_to_kappa_1e12(rq, prec):
    # the three-term sketch in a batch (and the emulated tiers on top of it)
    # against the oracle, kappa log-uniform up to 1e12
    g = np.random.default_rng(30 + prec)
    ms = g.integers(600, 9000, 12)
    ns = g.choice([16, 48, 96, 128], 12)
    kap = 10.0 ** g.uniform(2, 12, 12)
    xs = [synth.svd_matrix(int(m), int(n), float(k), 850 + i) for i, (m, n, k) in enumerate(zip(ms, ns, kap))]
    Xs = [dev(x) for x in xs]
    Qb, Rb, st = rq.rclupp_factor_batched(Xs, algo=rq.ALGO_RCLUPP, seed=71, prec=prec)
    assert np.all(st == 0)
    for i, x in enumerate(xs):
        m, n = x.shape
        q_o, r_o, _ = oracle.rclupp(x, S=oracle.gaussian_sketch_matrix(2 * n, m, 71 + i))
        q, r = host(Qb[i]), host(Rb[i])
        assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0), i
        assert oracle.orthogonality(q) <= max(10 * oracle.orthogonality(q_o), 1e-13), i
        assert oracle.residual(x, q, r) <= max(10 * oracle.residual(x, q_o, r_o), 1e-13), i


# ------------------------------------------- asynchronous, caller-recorded ---

@pytest.mark.parametrize("algo", [0, 1, 3])
def test_batched_async_matches_the_synchronous_call(rq, algo):
    # the same kernels and launch shapes as the graph of rclupp_factor_batched,
    # enqueued straight on the stream: every Q and R bit for bit, and the
    # statuses on the device
    xs, _ = _batch(10, 77 + algo, nmax=96)
    X = [dev(x) for x in xs]
    qs, rs, st = rq.rclupp_factor_batched(X, algo=algo, seed=5)
    qa, ra, dst = rq.rclupp_factor_batched_async(X, algo=algo, seed=5)
    torch.cuda.synchronize()
    assert dst.dtype == torch.int32 and dst.device.type == "cuda"
    assert np.array_equal(dst.cpu().numpy(), st)
    for i in range(len(xs)):
        assert torch.equal(qa[i], qs[i]) and torch.equal(ra[i], rs[i]), i


@pytest.mark.parametrize("mode", ["global", "relaxed"])
def test_batched_async_recorded_in_a_caller_graph(rq, mode):
    # a caller captures the call into its own CUDA graph (the workspace sized
    # by an earlier call outside the capture); replays give the results of
    # direct calls, also after the inputs change in place
    xs, _ = _batch(8, 91, nmax=64)
    X = [dev(x) for x in xs]
    qa, ra, _ = rq.rclupp_factor_batched_async(X, seed=3)
    torch.cuda.synchronize()
    qg = [torch.full_like(q, float("nan")) for q in qa]
    rg = [torch.full_like(r, float("nan")) for r in ra]
    dst = torch.full((len(xs),), -1, dtype=torch.int32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode=mode):
        rq.rclupp_factor_batched_async(X, seed=3, Qs=qg, Rs=rg, d_status=dst)
    torch.cuda.synchronize()
    assert int(dst[0]) == -1  # recorded, not run
    g.replay()
    torch.cuda.synchronize()
    assert int(dst.abs().max()) == 0
    for i in range(len(xs)):
        assert torch.equal(qg[i], qa[i]) and torch.equal(rg[i], ra[i]), i
    # new inputs in the same buffers
    xs2, _ = _batch(8, 92, nmax=64)
    for i in range(len(xs)):
        X[i].copy_(dev(synth.svd_matrix(xs[i].shape[0], xs[i].shape[1], 1e3, 500 + i)))
    g.replay()
    q2, r2, st2 = rq.rclupp_factor_batched(X, seed=3)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), st2)
    for i in range(len(xs)):
        assert torch.equal(qg[i], q2[i]) and torch.equal(rg[i], r2[i]), i


def test_batched_async_refuses_to_grow_its_workspace_while_captured(rq):
    # a thread's first call has no workspace yet, and none can be allocated
    # inside a capture: RCLUPP_ERR_UNSUPPORTED, nothing enqueued, and the
    # capture ends cleanly; the same call outside a capture then runs
    import threading
    xs, _ = _batch(4, 93, nmax=32)
    X = [dev(x) for x in xs]
    torch.cuda.synchronize()
    out = {}

    def worker():
        try:
            rq.rclupp_get_batch_policy()  # this thread's handle, created outside the capture
            qs = [rq.empty_colmajor(x.shape[0], x.shape[1], "cuda") for x in xs]
            rs = [rq.empty_colmajor(x.shape[1], x.shape[1], "cuda") for x in xs]
            dst = torch.full((len(xs),), -1, dtype=torch.int32, device="cuda")
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                try:
                    rq.rclupp_factor_batched_async(X, seed=2, Qs=qs, Rs=rs, d_status=dst)
                except rq.RclupError as e:
                    out["err"] = e
            _, _, dst = rq.rclupp_factor_batched_async(X, seed=2, Qs=qs, Rs=rs, d_status=dst)
            torch.cuda.synchronize()
            out["status"] = dst.cpu().numpy()
        except Exception as e:  # pragma: no cover - reported below
            out["exc"] = e

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert "exc" not in out, out.get("exc")
    assert out["err"].status == rq.Status.ERR_UNSUPPORTED
    assert np.all(out["status"] == 0)
