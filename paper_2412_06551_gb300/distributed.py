"""Row-sharded RCLUPP and CholeskyQR2 over the ranks of torch.distributed.

Each rank holds a contiguous block of rows of X: rows ``row0 .. row0 + m_r - 1``
of the m x n matrix, on its own GPU.  Every tall pass runs on the rank's own
rows; the only exchange is the sum of the partial s x n sketch and of the
partial n x n Gram matrices (the communication-avoiding property of
Section 1): RCLUPP needs three all-reduces (S X, Q1^T Q1, Q2^T Q2),
CholeskyQR2 two.  The small factorizations (sketch LU, Householder R,
Cholesky, triangular products) run replicated on every rank from identical
inputs, so every rank ends with the same R and its own rows of Q.  A rank
without rows (more ranks than rows) adds zero partials and returns an empty
block of Q, so it still takes part in every all-reduce.

RCLUPPr and LC2 are not sharded: their tall LU with partial pivoting needs an
argmax across all ranks for every column and the exchange of pivot rows.

The per-rank operations are those of this package's C ABI (:class:`LibrarySteps`);
the driver takes them, and the all-reduce, as parameters so that the
communication structure can be exercised with any implementation of the same
steps.
"""
from __future__ import annotations

from typing import Callable, Optional

from . import (SKETCH_GAUSSIAN, SKETCH_SRHT, RclupError, Status, rclupp_cholesky, rclupp_gram,
               rclupp_sketch, rclupp_sketch_precond, rclupp_trmm_upper, rclupp_trsm_gram)

__all__ = ["LibrarySteps", "torch_allreduce", "rclupp_factor_sharded", "cholqr2_factor_sharded",
           "row_block"]


def row_block(m: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous row block of `rank` among `world` ranks: (row0, rows)."""
    base, extra = divmod(m, world)
    row0 = rank * base + min(rank, extra)
    return row0, base + (1 if rank < extra else 0)


class LibrarySteps:
    """The per-rank steps on the rank's GPU through the C ABI."""

    def sketch(self, A, *, s, kind, zeta, seed, row0, order_log2=0):
        return rclupp_sketch(A, s=s, kind=kind, zeta=zeta, seed=seed, row0=row0, order_log2=order_log2)

    def precond(self, Y):
        return rclupp_sketch_precond(Y)

    def trsm_gram(self, A, R, *, gram):
        return rclupp_trsm_gram(A, R, gram=gram)

    def gram(self, A):
        return rclupp_gram(A)

    def cholesky(self, G):
        R, st, col = rclupp_cholesky(G, check=False)
        return R, st, col

    def trmm(self, A, B):
        return rclupp_trmm_upper(A, B)

    def zeros(self, like, rows, cols):
        """Column-major rows x cols zeros on the device of `like`."""
        import torch
        return torch.zeros((cols, rows), dtype=torch.float64, device=like.device).t()


def torch_allreduce(group=None) -> Callable:
    """In-place sum over the ranks of `group` (torch.distributed: NCCL for
    CUDA tensors, gloo for CPU tensors).

    NCCL takes only contiguous tensors, while the library returns
    column-major matrices (transposed views of contiguous memory).  A sum is
    elementwise, so such a matrix is reduced in place through its contiguous
    alias; any other layout goes through a contiguous copy."""
    import torch.distributed as dist

    def reduce_(t):
        if t.is_contiguous():
            alias = t
        elif t.dim() == 2 and t.t().is_contiguous():
            alias = t.t()
        else:
            c = t.contiguous()
            dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
            t.copy_(c)
            return t
        dist.all_reduce(alias, op=dist.ReduceOp.SUM, group=group)
        return t
    return reduce_


def _cholesky_or_raise(steps, G, pass_no):
    R, st, col = steps.cholesky(G)
    if st != Status.OK:
        # every rank holds the same all-reduced G, so every rank raises here
        err = RclupError("cholesky (pass %d, column %d)" % (pass_no, col), st)
        err.column = col
        raise err
    return R


def _trsm_gram(steps, A, R, gram, empty):
    """This rank's Q = A R^{-1} and, if asked, its partial Gram Q^T Q; a rank
    without rows returns an empty Q and a zero partial."""
    if not empty:
        return steps.trsm_gram(A, R, gram=gram)
    n = A.shape[1]
    return steps.zeros(A, 0, n), (steps.zeros(A, n, n) if gram else None)


def rclupp_factor_sharded(X_local, row0: int, *, s: Optional[int] = None, kind: int = SKETCH_GAUSSIAN,
                          zeta: int = 8, seed: int = 0, steps=None, allreduce: Optional[Callable] = None,
                          group=None, order_log2: int = 0):
    """[Q_local, R] = RCLUPP(X) (Algorithm 6) with X split by rows over the
    ranks.  X_local: this rank's rows (row0 .. row0 + m_r - 1), column-major
    on the rank's GPU.  The generated sketch is the one the whole matrix
    would get (entry (r, i) depends on the global row i), so the result
    equals the single-GPU factorization up to the order of the sums.  The
    SRHT needs the whole matrix's Hadamard order: order_log2 = b with
    2^b >= m (every rank passes the same b)."""
    steps = steps or LibrarySteps()
    allreduce = allreduce or torch_allreduce(group)
    n = X_local.shape[1]
    s = 2 * n if s is None else s
    sk = dict(s=s, kind=kind, zeta=zeta, seed=seed, row0=row0)
    if kind == SKETCH_SRHT:
        if order_log2 <= 0:
            raise ValueError("the SRHT of a row-sharded matrix needs order_log2 = ceil(log2(m)) "
                             "of the whole matrix")
        sk["order_log2"] = order_log2
    empty = X_local.shape[0] == 0
    # X_s = S X as a sum of the ranks' partials (all-reduce 1)
    Y = allreduce(steps.zeros(X_local, s, n) if empty else steps.sketch(X_local, **sk))
    # on every rank: LU of X_s, Householder R of M, R1 = R0 N
    R1 = steps.precond(Y)
    # CholeskyQR2 of Q1 = X R1^{-1} (all-reduces 2 and 3)
    Q1, G1 = _trsm_gram(steps, X_local, R1, True, empty)
    R2 = _cholesky_or_raise(steps, allreduce(G1), 1)
    Q2, G2 = _trsm_gram(steps, Q1, R2, True, empty)
    R4 = _cholesky_or_raise(steps, allreduce(G2), 2)
    Q, _ = _trsm_gram(steps, Q2, R4, False, empty)
    R = steps.trmm(R4, steps.trmm(R2, R1))  # R3 = R2 R1 (C4), R = R4 R3 (C8)
    return Q, R


def cholqr2_factor_sharded(X_local, *, steps=None, allreduce: Optional[Callable] = None, group=None):
    """[Q_local, R] = CholeskyQR2(X) (Algorithm 2) with X split by rows over
    the ranks (two all-reduces of n x n Gram partials)."""
    steps = steps or LibrarySteps()
    allreduce = allreduce or torch_allreduce(group)
    n = X_local.shape[1]
    empty = X_local.shape[0] == 0
    R1 = _cholesky_or_raise(steps, allreduce(steps.zeros(X_local, n, n) if empty
                                             else steps.gram(X_local)), 1)
    Q1, G1 = _trsm_gram(steps, X_local, R1, True, empty)
    R2 = _cholesky_or_raise(steps, allreduce(G1), 2)
    Q, _ = _trsm_gram(steps, Q1, R2, False, empty)
    return Q, steps.trmm(R2, R1)
