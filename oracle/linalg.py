"""Dense/sparse FP64 primitives of the oracle (test infrastructure only)."""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def spmm(A: sp.csr_matrix | None, X: np.ndarray) -> np.ndarray:
    """Y = A X for a CSR matrix (``MatDotMultiVec``, Section 3.4); A None means identity."""
    if A is None:
        return np.array(X, dtype=np.float64, copy=True)
    return np.asarray(A @ X, dtype=np.float64)


def b_norms(X: np.ndarray, BX: np.ndarray) -> np.ndarray:
    """Column B-norms sqrt(x_j^T B x_j) given X and BX."""
    return np.sqrt(np.maximum(np.einsum("ij,ij->j", X, BX), 0.0))


def sym_eig(M: np.ndarray):
    """Eigen-decomposition of a symmetric matrix, ascending eigenvalues.

    Uses LAPACK through numpy on (M + M^T)/2; this plays the role of the
    paper's ``dsyevx`` call in STEP 3 (Section 3.2) and of the small "SVD"
    M = Q Lambda Q^T in Algorithm 3.
    """
    M = 0.5 * (M + M.T)
    w, Q = np.linalg.eigh(M)
    return w, Q


def residual_norms(A, B, X: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Relative residuals ||A x - lambda B x|| / (|lambda| ||B^{1/2} x||) (Section 4).

    The paper states this form for its generalized FEM problem and the
    absolute form ||A x - lambda x|| / ||x|| for B = I; the relative form is
    used for every pencil here (the configurations are all positive definite).
    """
    AX = spmm(A, X)
    BX = spmm(B, X)
    R = AX - BX * lam[None, :]
    bn = b_norms(X, BX)
    return np.linalg.norm(R, axis=0) / (np.abs(lam) * bn)
