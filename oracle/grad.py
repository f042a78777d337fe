"""Reference gradients of eigenvalues and eigenvector functionals -- test infrastructure only.

Not in the paper: standard first-order perturbation theory for the pencil
A(c) x = lambda B x with A(c) = sum_e c_e P_e^T Khat P_e (Q1 cells, see
``workloads.q1_var``) and B independent of c, eigenvectors B-normalised.

* eigenvalue:  d lambda_i / d c_e = (P_e x_i)^T Khat (P_e x_i).
* functional f_i(x_i) with gradient g_i = df_i/dx_i: the adjoint mu_i solves
      (A - lambda_i B) mu_i = (I - B x_i x_i^T) g_i,   x_i^T B mu_i = 0,
  and d f_i / d c_e = -(P_e mu_i)^T Khat (P_e x_i).
  mu_i = sum_{j<=k, j!=i} x_j (x_j^T g_i)/(lambda_j - lambda_i) + z, where z
  solves the same system restricted to span(x_1..x_k)^{perp_B}, on which
  A - lambda_i B is SPD when lambda_i < lambda_{k+1}; z comes from CG with a
  B-projection after every step.
* per-nonzero form: dL/dA_pq = sum_i w_i x_ip x_iq - (mu_ip x_iq + x_ip mu_iq)/2.
"""
from __future__ import annotations

import numpy as np

from .linalg import spmm


def q1_khat(h: float) -> np.ndarray:
    """8x8 trilinear cell stiffness h (k(x)m(x)m + m(x)k(x)m + m(x)m(x)k), local index a0*4+a1*2+a2."""
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
    return h * (np.kron(k1, np.kron(m1, m1)) + np.kron(m1, np.kron(k1, m1))
                + np.kron(m1, np.kron(m1, k1)))


def cell_nodes(N: int) -> np.ndarray:
    """(N+1)^3 x 8 node indices of every cell (-1 for Dirichlet boundary nodes)."""
    e = np.arange(N + 1)
    E0, E1, E2 = np.meshgrid(e, e, e, indexing="ij")
    out = np.empty(((N + 1) ** 3, 8), dtype=np.int64)
    for a0 in (0, 1):
        for a1 in (0, 1):
            for a2 in (0, 1):
                i0, i1, i2 = E0 + a0 - 1, E1 + a1 - 1, E2 + a2 - 1
                ok = (i0 >= 0) & (i0 < N) & (i1 >= 0) & (i1 < N) & (i2 >= 0) & (i2 < N)
                idx = np.where(ok, (i0 * N + i1) * N + i2, -1)
                out[:, a0 * 4 + a1 * 2 + a2] = idx.ravel()
    return out


def _gather(v: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    g = np.where(nodes >= 0, v[np.maximum(nodes, 0)], 0.0)
    return g


def cell_bilinear(N: int, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Per cell (P_e u)^T Khat (P_e v)."""
    nodes = cell_nodes(N)
    K = q1_khat(1.0 / (N + 1))
    ue = _gather(u, nodes)
    ve = _gather(v, nodes)
    return np.einsum("ea,ab,eb->e", ue, K, ve)


def projected_cg(A, B, lam_i: float, X: np.ndarray, rhs: np.ndarray, tol: float = 1e-12,
                 max_iter: int = 100000) -> np.ndarray:
    """Solve (A - lam_i B) z = rhs on span(X)^{perp_B}.

    With P = I - X X^T B, plain CG runs on the symmetric operator P^T (A - lam_i B) P
    with right-hand side P^T rhs; the answer is P z.
    """
    BX = spmm(B, X)

    def proj(v):                      # P = I - X X^T B
        return v - X @ (BX.T @ v)

    def projT(v):                     # P^T = I - B X X^T
        return v - BX @ (X.T @ v)

    def op(v):
        u = proj(v)
        return projT(spmm(A, u[:, None])[:, 0] - lam_i * spmm(B, u[:, None])[:, 0])

    b = projT(rhs)
    z = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bn = np.sqrt(rr)
    for _ in range(max_iter):
        if np.sqrt(rr) <= tol * bn or bn == 0.0:
            break
        q = op(p)
        alpha = rr / float(p @ q)
        z = z + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return proj(z)


def adjoint(A, B, lam: np.ndarray, X: np.ndarray, i: int, g: np.ndarray, tol: float = 1e-12):
    """mu_i for functional gradient g (deflation of X's columns plus projected CG)."""
    BXg = X.T @ g
    mu = np.zeros(X.shape[0])
    for j in range(X.shape[1]):
        if j != i:
            mu += X[:, j] * (BXg[j] / (lam[j] - lam[i]))
    rhs = g - spmm(B, X) @ (X.T @ g)           # (I - B X X^T) g: component outside span(X)
    mu += projected_cg(A, B, lam[i], X, rhs, tol)
    return mu


def loss_grad_cells(N: int, A, B, lam: np.ndarray, X: np.ndarray, w_lam: np.ndarray,
                    G_x: np.ndarray | None, tol: float = 1e-12) -> np.ndarray:
    """dL/dc for L = sum_i w_lam_i lambda_i + sum_i f_i(x_i), G_x[:, i] = df_i/dx_i."""
    g = np.zeros((N + 1) ** 3)
    for i in range(X.shape[1]):
        g += w_lam[i] * cell_bilinear(N, X[:, i], X[:, i])
        if G_x is not None and np.any(G_x[:, i]):
            mu = adjoint(A, B, lam, X, i, G_x[:, i], tol)
            g -= cell_bilinear(N, mu, X[:, i])
    return g


def loss_grad_nonzeros(A, lam: np.ndarray, X: np.ndarray, w_lam: np.ndarray,
                       MU: np.ndarray | None) -> np.ndarray:
    """dL/dA on the CSR nonzeros of A (symmetrised adjoint term)."""
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    cols = A.indices
    out = np.zeros(A.nnz)
    for i in range(X.shape[1]):
        out += w_lam[i] * X[rows, i] * X[cols, i]
        if MU is not None:
            out -= 0.5 * (MU[rows, i] * X[cols, i] + X[rows, i] * MU[cols, i])
    return out
