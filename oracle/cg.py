"""STEP 6 of Algorithm 1: the shifted inexact inverse-power solve (test infrastructure only).

For each column j of the active block X_n the system
    (A - theta B) w_j = (lambda_j - theta) B x_j            (Eq. compW)
is solved approximately by plain conjugate gradients from the initial guess
w_j = x_j.  Columns are independent (the paper says only "some CG steps";
reading: column-wise CG with one common theta).  Each column stops when
||r|| <= rtol ||r_0|| or after max_iter iterations (Section 4.1: 1 % and 30),
or at a breakdown p^T (A - theta B) p <= 0, keeping its current iterate.
The shifted matrix is formed explicitly, as Section 4.1 recommends.

Preconditioned variant (``precond=True``): Section 2 suggests a preconditioner for
STEP 6 (algebraic multigrid, for discretised PDEs).  Here the preconditioner is the
diagonal M = |diag(A - theta B)| (Jacobi) of the same shifted system, with the same
shift; the standard preconditioned CG recurrences use r^T M^-1 r in alpha and beta,
and the stop test stays on the unpreconditioned ||r||.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .linalg import spmm


def shifted_matrix(A, B, theta: float):
    """S = A - theta B as an explicit CSR matrix (B None means identity)."""
    if theta == 0.0:
        return A
    Bm = sp.identity(A.shape[0], format="csr") if B is None else B
    return (A - theta * Bm).tocsr()


def jacobi_inverse(S) -> np.ndarray:
    """1 / |diag(S)| (zero entries of the diagonal are left unscaled)."""
    d = np.abs(S.diagonal())
    return np.where(d > 0.0, 1.0 / np.where(d > 0.0, d, 1.0), 1.0)


def shifted_cg(A, B, theta: float, X: np.ndarray, lam: np.ndarray, max_iter: int = 30,
               rtol: float = 1e-2, rhs: np.ndarray | None = None, precond: bool = False):
    """Return (W, iterations per column, breakdown flags).

    ``rhs`` overrides the right-hand side (default (lambda_j - theta) B x_j).
    All columns advance together but every scalar (alpha, beta, the stop
    test) is per column, so the result equals k independent CG runs.
    """
    n, k = X.shape
    if rhs is None:
        rhs = spmm(B, X) * (np.asarray(lam) - theta)[None, :]
    S = shifted_matrix(A, B, theta)
    minv = jacobi_inverse(S)[:, None] if precond else 1.0
    x = np.array(X, dtype=np.float64, copy=True)
    r = rhs - spmm(S, x)
    z = r * minv
    p = z.copy()
    rr = np.einsum("ij,ij->j", r, r)
    rz = np.einsum("ij,ij->j", r, z)
    r0 = np.sqrt(rr)
    active = np.ones(k, dtype=bool)
    iters = np.zeros(k, dtype=np.int64)
    broke = np.zeros(k, dtype=bool)
    for _ in range(max_iter):
        active &= ~(np.sqrt(rr) <= rtol * r0)
        if not active.any():
            break
        q = spmm(S, p)
        pq = np.einsum("ij,ij->j", p, q)
        bad = active & ~(pq > 0.0)
        broke |= bad
        active &= ~bad
        if not active.any():
            break
        alpha = np.where(active, rz / np.where(active, pq, 1.0), 0.0)
        x += p * alpha[None, :]
        r -= q * alpha[None, :]
        z = r * minv
        rr_new = np.einsum("ij,ij->j", r, r)
        rz_new = np.einsum("ij,ij->j", r, z)
        beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
        p = np.where(active[None, :], z + p * beta[None, :], p)
        rr = np.where(active, rr_new, rr)
        rz = np.where(active, rz_new, rz)
        iters += active
    return x, iters, broke
