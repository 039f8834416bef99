"""Pins for the oracle's subsampled randomized Hadamard transform (SRHT), one
of the common sketches of Section 3.  The Hadamard structure is checked
against scipy's Sylvester construction (a Kronecker product, not the popcount
formula the oracle uses) and against an independent fast Walsh-Hadamard
transform; the sampling against the permutation property; the scale against
exact orthogonality at full sampling and the expected squared norm; the signs
against the Philox words (Philox itself is pinned by its published test
vectors).  No GPU is used."""
import numpy as np
import pytest
import scipy.linalg

import oracle


def _fwht_rows(a):
    """Unnormalised Walsh-Hadamard transform along axis 0 (length 2^b) by
    butterflies in natural (Sylvester) order."""
    a = np.array(a, dtype=np.float64, copy=True)
    h = 1
    while h < a.shape[0]:
        a = a.reshape((-1, 2, h) + a.shape[1:])
        top, bot = a[:, 0].copy(), a[:, 1].copy()
        a[:, 0], a[:, 1] = top + bot, top - bot
        a = a.reshape((-1,) + a.shape[3:])
        h *= 2
    return a


@pytest.mark.parametrize("s,m,row0,seed", [(1, 1, 0, 0), (2, 2, 0, 5), (4, 6, 0, 7), (8, 37, 0, 11),
                                           (16, 100, 28, 3), (64, 64, 0, 2**40 + 9),
                                           (12, 200, 313, 17)])
def test_dense_is_sampled_sylvester_hadamard(s, m, row0, seed):
    b = oracle.srht_order_log2(row0 + m)
    S = oracle.srht_dense(s, m, seed, b=b, row0=row0)
    H = scipy.linalg.hadamard(1 << b).astype(np.float64)
    p = oracle.srht_perm(s, b, seed)
    d = oracle.srht_signs(m, seed, row0).astype(np.float64)
    ref = H[p][:, row0:row0 + m] * d[None, :] / np.sqrt(s)
    np.testing.assert_array_equal(S, ref)


@pytest.mark.parametrize("b", list(range(0, 13)))
def test_perm_is_a_bijection(b):
    for seed in (0, 1, 12345):
        p = oracle.srht_perm(1 << b, b, seed)
        assert np.array_equal(np.sort(p), np.arange(1 << b))


def test_perm_depends_on_seed_and_order():
    a = oracle.srht_perm(64, 10, 1)
    assert not np.array_equal(a, oracle.srht_perm(64, 10, 2))
    assert not np.array_equal(a, oracle.srht_perm(64, 11, 1) % 1024)


def test_perm_first_row_is_roughly_uniform():
    # p_0 over 4000 seeds at b = 4: each of the 16 rows about 250 times
    counts = np.bincount([oracle.srht_perm(1, 4, seed)[0] for seed in range(4000)], minlength=16)
    assert counts.min() > 170 and counts.max() < 330


def test_signs_follow_philox_words():
    seed = 0x1234_5678_9ABC
    d = oracle.srht_signs(300, seed, row0=1000)
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for i in range(300):  # every bit position k = 0..127, across three Philox blocks
        g = 1000 + i
        q = g >> 7
        w = oracle.philox4x32_10(np.array([q & 0xFFFFFFFF, q >> 32, 0, 0x53524844], dtype=np.uint32), key)
        k = g & 127
        bit = (int(w[k >> 5]) >> (k & 31)) & 1
        assert d[i] == (-1 if bit else 1)
    big = oracle.srht_signs(200000, 3)
    assert abs(big.astype(np.float64).mean()) < 0.01


def test_row_block_is_slice_of_whole():
    full = oracle.srht_dense(24, 300, 9, b=9)
    part = oracle.srht_dense(24, 77, 9, b=9, row0=150)
    np.testing.assert_array_equal(part, full[:, 150:227])


@pytest.mark.parametrize("m,s,n", [(37, 8, 3), (64, 20, 5), (200, 33, 4)])
def test_sketch_equals_fast_transform(m, s, n):
    g = np.random.default_rng(m + s)
    x = g.standard_normal((m, n))
    seed = 77
    b = oracle.srht_order_log2(m)
    y = oracle.sketch_dense(oracle.srht_dense(s, m, seed), x)
    dx = np.zeros((1 << b, n))
    dx[:m] = oracle.srht_signs(m, seed)[:, None] * x
    ref = _fwht_rows(dx)[oracle.srht_perm(s, b, seed)] / np.sqrt(s)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-13 * np.abs(x).sum())


def test_full_sampling_is_orthogonal():
    # s = m = m': S = H D / sqrt(m) with rows permuted is orthogonal
    S = oracle.srht_dense(128, 128, 4)
    np.testing.assert_allclose(S.T @ S, np.eye(128), rtol=0, atol=1e-14)
    x = np.random.default_rng(1).standard_normal(128)
    assert abs(np.linalg.norm(S @ x) - np.linalg.norm(x)) < 1e-13


def test_expected_squared_norm_is_preserved():
    # E ||S x||^2 = ||x||^2 over the draws of R and D (scale 1/sqrt(s), not 1/sqrt(m'))
    x = np.random.default_rng(2).standard_normal(100)
    vals = [np.linalg.norm(oracle.srht_dense(16, 100, seed) @ x) ** 2 for seed in range(300)]
    assert abs(np.mean(vals) / np.dot(x, x) - 1.0) < 0.05


def test_subspace_embedding():
    # a 2n-row SRHT of an orthonormal basis keeps its singular values near 1
    g = np.random.default_rng(3)
    q, _ = np.linalg.qr(g.standard_normal((4096, 16)))
    sv = np.linalg.svd(oracle.sketch_dense(oracle.srht_dense(64, 4096, 5), q), compute_uv=False)
    assert sv.min() > 0.4 and sv.max() < 1.6


def test_rclupp_with_srht_sketch():
    g = np.random.default_rng(4)
    m, n = 300, 12
    u, _ = np.linalg.qr(g.standard_normal((m, n)))
    v, _ = np.linalg.qr(g.standard_normal((n, n)))
    x = u @ np.diag(np.logspace(0, -8, n)) @ v.T
    q, r, st = oracle.rclupp(x, S=oracle.srht_dense(2 * n, m, 6))
    assert st == 0
    assert oracle.orthogonality(q) < 1e-14
    assert oracle.residual(x, q, r) < 1e-15


def test_selected_rows_are_rows_of_whole():
    full = oracle.srht_dense(40, 123, 8)
    rows = [0, 7, 39, 12]
    np.testing.assert_array_equal(oracle.srht_dense_rows(rows, 40, 123, 8), full[rows])
