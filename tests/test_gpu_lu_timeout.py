"""Failure detection of the tall LU's bounded device wait, through the C ABI.

A panel of the tall LU runs as one cooperative launch whose CTAs meet at a
grid-wide barrier after each pivot selection.  The test arms the library's
one-shot fault (the first barrier expects one arrival more than the grid
has, a flag nothing will set), with a 50 ms limit: the wait must run out,
the call must return RCLUPP_ERR_TIMEOUT naming the LU step and the column
whose pivot was awaited, and the same handle must then factor correctly
(pivot rows bit-exact against the oracle's GEPP).  Nothing faults, traps or
hangs: every wait is bounded and the kernel returns after it.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ERR_TIMEOUT = -6
FAULT_LU_BARRIER_STALL = 1


def _colmajor(x):
    return torch.from_numpy(np.ascontiguousarray(np.asfortranarray(x).T)).to("cuda").t()


@pytest.fixture()
def lib_and_handle():
    import paper_2412_06551_gb300 as rq
    lib = rq.load()
    h = ctypes.c_void_p()
    assert lib.rclupp_create(ctypes.byref(h), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    yield lib, h
    lib.rclupp_destroy(h)


def _lu(lib, h, x):
    m, n = x.shape
    A = _colmajor(x)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    col = ctypes.c_int64(-2)
    st = lib.rclupp_tall_lupp(h, m, n, ctypes.c_void_p(A.data_ptr()), A.stride(1),
                              ctypes.c_void_p(ipiv.data_ptr()), ctypes.byref(col))
    torch.cuda.synchronize()
    return st, int(col.value), A, ipiv


def test_lu_barrier_wait_runs_out_and_the_handle_recovers(lib_and_handle):
    lib, h = lib_and_handle
    x = synth.svd_matrix(20000, 24, 1e3, 5)
    assert lib.rclupp_set_wait_limit(h, 50_000_000) == 0
    assert lib.rclupp_inject_fault(h, FAULT_LU_BARRIER_STALL) == 0
    st, col, _, _ = _lu(lib, h, x)
    assert st == ERR_TIMEOUT and col == 1, (st, col)
    # the injection was one-shot and the handle is usable: a full LU now
    st, col, A, ipiv = _lu(lib, h, x)
    assert st == 0 and col == -1
    _, ipiv_o, st_o, _ = oracle.gepp(x)
    assert st_o == 0 and np.array_equal(ipiv.cpu().numpy(), np.asarray(ipiv_o))
    assert lib.rclupp_set_wait_limit(h, 0) == 0


def test_rcluppr_reports_the_timeout_and_recovers(lib_and_handle):
    import paper_2412_06551_gb300 as rq
    lib, h = lib_and_handle
    m, n = 12000, 40
    x = synth.svd_matrix(m, n, 1e6, 6)
    X = _colmajor(x)
    opts = rq.Opts()
    opts.kind, opts.s, opts.seed, opts.prec, opts.zeta = 0, 2 * n, 3, 0, 8
    info = rq.Info()

    def run():
        Q = torch.empty((n, m), dtype=torch.float64, device="cuda").t()
        R = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
        st = lib.rclupp_r_factor(h, m, n, ctypes.c_void_p(X.data_ptr()), X.stride(1), ctypes.byref(opts),
                                 ctypes.c_void_p(Q.data_ptr()), Q.stride(1), ctypes.c_void_p(R.data_ptr()),
                                 R.stride(1), ctypes.byref(info))
        return st, Q, R

    assert lib.rclupp_set_wait_limit(h, 50_000_000) == 0
    assert lib.rclupp_inject_fault(h, FAULT_LU_BARRIER_STALL) == 0
    st, _, _ = run()
    assert st == ERR_TIMEOUT and info.failed_step == 2 and info.info == 1
    st, Q, R = run()
    assert st == 0
    q, r = Q.cpu().numpy(), R.cpu().numpy()
    q_o, r_o, _ = oracle.rcluppr(x, S=oracle.gaussian_sketch_matrix(2 * n, m, 3))
    assert oracle.orthogonality(q) <= max(10 * oracle.orthogonality(q_o), 1e-13)
    assert oracle.residual(x, q, r) <= max(10 * oracle.residual(x, q_o, r_o), 1e-13)


def test_fault_argument_is_checked(lib_and_handle):
    lib, h = lib_and_handle
    assert lib.rclupp_inject_fault(h, 7) == -1
    assert lib.rclupp_inject_fault(h, 0) == 0
