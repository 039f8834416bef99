"""The allocation-free Gram entry point (rclupp_gram_noalloc), called through
the C ABI, against the allocating one (rclupp_gram).

rclupp_gram_noalloc serves callers that cannot let the library allocate
device memory; it keeps its scratch in a fixed array inside the library.
Two calls in a row on different shapes check that what the previous call
left in that shared array does not leak into the next result.  Each result
is compared with the allocating entry point and with the CPU oracle's Gram
(sequential sums).  The tolerance is the one the Gram parity tests use: two
sums of the same m products in different orders differ by at most
2 gamma_m (|A|^T |A|).
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _gamma(k):
    return k * U / (1 - k * U)


def _dev(a):
    a = np.asfortranarray(a)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda").t()


def _noalloc(lib, A, m, n):
    G = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda").t()
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.rclupp_gram_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), A.stride(1),
                                 ctypes.c_void_p(G.data_ptr()), G.stride(1), ctypes.c_void_p(stream))
    return st, G


def _reference(lib, A, m, n):
    h = ctypes.c_void_p()
    assert lib.rclupp_create(ctypes.byref(h), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    G = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    st = lib.rclupp_gram(h, m, n, ctypes.c_void_p(A.data_ptr()), A.stride(1), 0,
                         ctypes.c_void_p(G.data_ptr()), G.stride(1))
    lib.rclupp_destroy(h)
    assert st == 0
    return G


def test_noalloc_gram_matches_allocating_gram_twice():
    import paper_2412_06551_gb300 as rq
    lib = rq.load()
    for (m, n, seed) in ((100003, 128, 1), (5000, 40, 2)):
        x = synth.svd_matrix(m, n, 1e4, seed)
        A = _dev(x)
        st, G = _noalloc(lib, A, m, n)
        assert st == 0
        G_ref = _reference(lib, A, m, n)
        g, g_ref = G.cpu().numpy(), G_ref.cpu().numpy()
        tol = 2 * _gamma(m) * (np.abs(x).T @ np.abs(x))
        assert np.all(np.isfinite(g))
        assert np.all(np.abs(g - g_ref) <= tol)
        g_orc = oracle.gram(x)
        assert np.all(np.abs(g - g_orc) <= tol)


def test_noalloc_gram_rejects_sizes_beyond_its_limit():
    import paper_2412_06551_gb300 as rq
    lib = rq.load()
    A = torch.zeros((200, 129), dtype=torch.float64, device="cuda").t().t()
    A = A.t().contiguous().t()
    st, _ = _noalloc(lib, A, 200, 129)
    assert st == rq.Status.ERR_UNSUPPORTED
