"""Degenerate inputs through every driver, on the GPU, through the C ABI.

The paper assumes a finite X of full column rank (Section 1); outside that
set the library reports a status instead of returning NaN-filled factors.

* A zero column (rank n - 1): every quantity touching it is an exact zero,
  so the failing step and column are determined and equal the oracle's.
  RCLUPP's sketch S X has a zero column, so the small LU of Algorithm 6 finds
  a zero pivot there; RCLUPPr and LC2 find it in the tall LU of X
  (Algorithms 7 and 4); CholeskyQR2 (Algorithm 2) meets a zero radicand in
  the first Cholesky; RCholeskyQR (Algorithm 5) and SCholeskyQR3 (Algorithm
  3) get a zero (or undefined) column of Q1 and break down in the Cholesky of
  its Gram.  The oracle reports the same statuses and columns (its info packs
  the CholeskyQR pass p as 100000 p + column).
* A NaN or an infinity: the device LU pivot searches ignore NaN candidates
  and report RCLUPP_ERR_NONFINITE when a column has no finite non-zero
  candidate left; otherwise the non-finite values reach a Gram and the
  Cholesky reports a breakdown.  The oracle's LU has no such check (a NaN
  pivot runs on until its Cholesky breaks down), so only the exact cases are
  compared column for column; every other case must end in one of these two
  numerical statuses, never in RCLUPP_OK.
* After any failure the handle keeps working: the next factorization on a
  finite matrix passes the usual gate.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M, N, S = 3000, 24, 48
DRIVERS = ["rclupp", "rcluppr", "cholqr2", "lc2", "rcholqr", "scholqr3"]
RANDOMIZED = {"rclupp", "rcluppr", "rcholqr"}
# failed_step of the zero-column breakdown: 1 sketch LU, 2 tall LU, 3 first
# Cholesky of the CholeskyQR passes
ZERO_COL_STEP = {"rclupp": 1, "rcluppr": 2, "lc2": 2, "cholqr2": 3, "rcholqr": 3, "scholqr3": 3}


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


def _fn(rq, name):
    return {"rclupp": rq.rclupp_factor, "rcluppr": rq.rclupp_r_factor, "cholqr2": rq.cholqr2_factor,
            "lc2": rq.lc2_factor, "rcholqr": rq.rcholqr_factor, "scholqr3": rq.scholqr3_factor}[name]


def _call(rq, name, X, **kw):
    if name in RANDOMIZED:
        kw.setdefault("s", S)
        kw.setdefault("seed", 3)
        return _fn(rq, name)(X, **kw)
    return _fn(rq, name)(X)


def _base():
    return synth.svd_matrix(M, N, 1e4, 21)


def _still_works(rq, name):
    x = _base()
    Q, R, _ = _call(rq, name, dev(x))
    q, r = host(Q), host(R)
    assert oracle.orthogonality(q) <= 1e-13 and oracle.residual(x, q, r) <= 1e-13
    assert np.array_equal(r, np.triu(r)) and np.all(np.diag(r) > 0)


@pytest.mark.parametrize("name", DRIVERS)
def test_zero_column_status_matches_oracle(rq, name):
    x = _base()
    x[:, 7] = 0.0
    with pytest.raises(rq.RclupError) as e:
        _call(rq, name, dev(x))
    st, info = e.value.status, e.value.info
    with pytest.raises(oracle.OracleError) as eo:
        if name in RANDOMIZED:
            getattr(oracle, name)(x, S=oracle.gaussian_sketch_matrix(S, M, 3))
        else:
            getattr(oracle, name)(x)
    assert st == eo.value.status, (st, eo.value.status)
    assert info.failed_step == ZERO_COL_STEP[name] and info.info == 7, (info.failed_step, info.info)
    o_pass, o_col = divmod(eo.value.info, 100000)
    assert o_col == 7
    if o_pass:  # the oracle's CholeskyQR pass p is the device's failed_step 2 + p
        assert info.failed_step == 2 + o_pass
    _still_works(rq, name)


@pytest.mark.parametrize("value", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("name", DRIVERS)
def test_nonfinite_entry_gives_a_numerical_status(rq, name, value):
    x = _base()
    x[5, 4] = value
    with pytest.raises(rq.RclupError) as e:
        _call(rq, name, dev(x))
    assert e.value.status in (rq.Status.ERR_NONFINITE, rq.Status.ERR_CHOL_BREAKDOWN), e.value
    _still_works(rq, name)


def test_nan_in_sketch_is_caught_by_the_sketch_lu(rq):
    # every entry of column 4 of S X is NaN, so the small LU of Algorithm 6
    # has no pivot candidate in column 4
    x = _base()
    x[5, 4] = np.nan
    with pytest.raises(rq.RclupError) as e:
        _call(rq, "rclupp", dev(x))
    assert e.value.status == rq.Status.ERR_NONFINITE
    assert (e.value.info.failed_step, e.value.info.info) == (1, 4)


@pytest.mark.parametrize("value", [np.nan, np.inf])
def test_cholqr2_nonfinite_breaks_down_where_the_oracle_does(rq, value):
    x = _base()
    x[5, 4] = value
    with pytest.raises(rq.RclupError) as e:
        _call(rq, "cholqr2", dev(x))
    with pytest.raises(oracle.OracleError) as eo:
        oracle.cholqr2(x)
    assert e.value.status == eo.value.status == rq.Status.ERR_CHOL_BREAKDOWN
    assert (e.value.info.failed_step, e.value.info.info) == (3, eo.value.info) == (3, 4)


def test_batched_poisoned_problem_leaves_the_others_alone(rq):
    xs = [synth.svd_matrix(2000 + 500 * i, 16 + 8 * i, 1e6, 60 + i) for i in range(4)]
    xs[2][11, 3] = np.nan
    Xs = [dev(x) for x in xs]
    Qb, Rb, st = rq.rclupp_factor_batched(Xs, seed=40, check=False)
    assert st[2] in (rq.Status.ERR_NONFINITE, rq.Status.ERR_CHOL_BREAKDOWN), st
    for i in (0, 1, 3):
        assert st[i] == 0, st
        q, r, _ = rq.rclupp_factor(Xs[i], s=2 * xs[i].shape[1], seed=40 + i)
        assert torch.equal(Qb[i], q) and torch.equal(Rb[i], r), i
