"""STEP 2 of Algorithm 1: B-orthogonalisation of the new block W (test infrastructure only).

Two phases, as Section 3.1 describes:

1. deflation against an already B-orthonormal block Q = [X, P]:
   W <- W - Q (Q^T B W), repeated until Q^T B W is small relative to the
   columns of W (the first loop of Algorithm 2; the paper's "small enough");
2. Algorithm 3, RecursiveOrthSVD: split the columns in halves, orthonormalise
   the left half recursively, deflate the right half against it
   (R = (B X_left)^T X_right, X_right -= X_left R, repeated), recurse on the
   right half; a leaf of at most c = min(m, 16) columns is orthonormalised by
   M = X^T B X = Q Lambda Q^T, X <- X Q Lambda^{-1/2}, repeated until
   Lambda ~ I (two or three times).

Readings where the paper is silent (collected in ``OrthParams``):
* W is scaled to unit B-norm columns before phase 1, so every "small" test
  below is relative to that unit start;
* "small enough" for a deflation step means max_ij |R_ij| / ||w_j||_B <= tol,
  measured on the block before the subtraction, at most three passes;
* a column whose B-norm after phase 1 fell below ``drop_tol`` is linearly
  dependent on Q and is removed; inside a leaf an eigenvalue of M "close to
  zero" is one at or below max(leaf_rel * max(Lambda), leaf_drop): relative to
  the rounding level of the computed Gram M, with an absolute floor for a block
  whose columns all collapsed; such directions are removed.  Removal
  compacts the block (the paper moves the trailing vectors into the freed
  slots; only the span matters to the Rayleigh-Ritz step);
* when the column count m is not a power of two the split is at floor(m/2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .linalg import spmm, b_norms, sym_eig


@dataclass
class OrthParams:
    defl_tol: float = 1e-12
    defl_max: int = 3
    drop_tol: float = 1e-13
    leaf_tol: float = 1e-12
    leaf_max: int = 3
    leaf_drop: float = 1e-20
    leaf_rel: float = 1e-14
    inner_tol: float = 1e-12
    inner_max: int = 3
    leaf: int = 16


def normalize_cols(W: np.ndarray, BW: np.ndarray, tiny: float = 1e-300):
    """Scale columns to unit B-norm, removing exactly-zero columns."""
    s = b_norms(W, BW)
    keep = s > tiny
    return W[:, keep] / s[keep], BW[:, keep] / s[keep]


def deflate_against(W: np.ndarray, Q: np.ndarray, B, p: OrthParams = OrthParams()):
    """B-orthogonalise W against the B-orthonormal block Q; returns (W, BW).

    W is first scaled to unit B-norm columns; then W <- W - Q (Q^T B W) is
    repeated until the relative size of Q^T B W is below ``defl_tol`` (at most
    ``defl_max`` passes); columns left with B-norm <= ``drop_tol`` are dropped
    and the rest are rescaled to unit B-norm.
    """
    BW = spmm(B, W)
    W, BW = normalize_cols(W, BW)
    if Q is not None and Q.shape[1] > 0 and W.shape[1] > 0:
        for _ in range(p.defl_max):
            R = Q.T @ BW
            s = b_norms(W, BW)
            crit = float(np.max(np.abs(R) / s[None, :]))
            W = W - Q @ R
            BW = spmm(B, W)
            if crit <= p.defl_tol:
                break
        s = b_norms(W, BW)
        keep = s > p.drop_tol
        W = W[:, keep] / s[keep]
        BW = BW[:, keep] / s[keep]
    return W, BW


def _leaf(W: np.ndarray, BW: np.ndarray, p: OrthParams):
    for _ in range(p.leaf_max):
        if W.shape[1] == 0:
            break
        M = W.T @ BW
        lam, Q = sym_eig(M)
        keep = lam > max(p.leaf_rel * float(np.max(lam)), p.leaf_drop)
        C = Q[:, keep] / np.sqrt(lam[keep])[None, :]
        W = W @ C
        BW = BW @ C
        if keep.any() and float(np.max(np.abs(lam[keep] - 1.0))) <= p.leaf_tol:
            break
    return W, BW


def _recursive(W: np.ndarray, BW: np.ndarray, c: int, p: OrthParams):
    length = W.shape[1]
    if length == 0:
        return W, BW
    if length <= c:
        return _leaf(W, BW, p)
    h = length // 2
    L, BL = _recursive(W[:, :h], BW[:, :h], c, p)
    Rt, BRt = W[:, h:], BW[:, h:]
    if L.shape[1] > 0:
        for _ in range(p.inner_max):
            R = BL.T @ Rt
            s = np.maximum(b_norms(Rt, BRt), 1e-300)
            crit = float(np.max(np.abs(R) / s[None, :]))
            Rt = Rt - L @ R
            BRt = BRt - BL @ R
            if crit <= p.inner_tol:
                break
    Rt, BRt = _recursive(Rt, BRt, c, p)
    return np.hstack([L, Rt]), np.hstack([BL, BRt])


def recursive_orth_svd(W: np.ndarray, BW: np.ndarray, p: OrthParams = OrthParams()):
    """Algorithm 3 on all columns of W (with BW = B W); returns (W, BW) B-orthonormal."""
    c = min(W.shape[1], p.leaf)
    return _recursive(W, BW, max(c, 1), p)


def b_orthonormalize(W: np.ndarray, Q: np.ndarray | None, B, p: OrthParams = OrthParams()):
    """STEP 2 for the new block: deflate against Q then Algorithm 3."""
    W, BW = deflate_against(W, Q, B, p)
    return recursive_orth_svd(W, BW, p)


def _mgs_block(X: np.ndarray, BX: np.ndarray, p: OrthParams):
    """Modified Gram-Schmidt inside one block in the B inner product (Algorithm 2's
    per-block step): column j is scaled to unit B-norm and removed from every later
    column of the block at once.  A column whose B-norm has fallen to ``drop_tol``
    (the columns start Algorithm 2 at unit B-norm) is linearly dependent: it is
    removed and the block's rearmost column takes its place (Section 3.1).  The pass
    is repeated while the block's Gram differs from I by more than ``leaf_tol`` (at
    most ``leaf_max`` passes), as the "small enough" loops of Algorithm 2 are."""
    X, BX = X.copy(), BX.copy()
    for _ in range(p.leaf_max):
        m = X.shape[1]
        j = 0
        while j < m:
            s = float(np.sqrt(max(X[:, j] @ BX[:, j], 0.0)))
            if s <= p.drop_tol:
                X[:, j], BX[:, j] = X[:, m - 1], BX[:, m - 1]
                m -= 1
                continue
            X[:, j] /= s
            BX[:, j] /= s
            r = X[:, j + 1:m].T @ BX[:, j]
            X[:, j + 1:m] -= np.outer(X[:, j], r)
            BX[:, j + 1:m] -= np.outer(BX[:, j], r)
            j += 1
        X, BX = X[:, :m], BX[:, :m]
        if m == 0 or float(np.max(np.abs(X.T @ BX - np.eye(m)))) <= p.leaf_tol:
            break
    return X, BX


def modified_block_orth(X: np.ndarray, X0: np.ndarray | None, B, b: int | None = None,
                        p: OrthParams = OrthParams()):
    """Algorithm 2 (modified block orthogonalisation), block size b = min(m/4, 200).

    Deflation against X0 as in ``deflate_against``; then for k = 1..l: the block
    X_k is orthonormalised by modified Gram-Schmidt (``_mgs_block``), and all later
    blocks together are deflated against it, R = [X_{k+1},...,X_l]^T (B X_k),
    X_rest -= X_k R^T, repeated until R is small relative to the columns.
    """
    X, BX = deflate_against(X, X0, B, p)
    m = X.shape[1]
    if b is None:
        b = max(1, min(m // 4, 200))
    done, Bdone = [], []
    rest, Brest = X, BX
    while rest.shape[1] > 0:
        Xk, BXk = _mgs_block(rest[:, :b], Brest[:, :b], p)
        done.append(Xk)
        Bdone.append(BXk)
        rest, Brest = rest[:, b:], Brest[:, b:]
        if rest.shape[1] == 0 or Xk.shape[1] == 0:
            continue
        for _ in range(p.inner_max):
            R = rest.T @ BXk
            s = np.maximum(b_norms(rest, Brest), 1e-300)
            crit = float(np.max(np.abs(R) / s[:, None]))
            rest = rest - Xk @ R.T
            Brest = Brest - BXk @ R.T
            if crit <= p.inner_tol:
                break
    return np.hstack(done), np.hstack(Bdone)


def b_orthonormalize_alg2(W: np.ndarray, Q: np.ndarray | None, B, p: OrthParams = OrthParams()):
    """STEP 2 with Algorithm 2 in place of Algorithm 3 (the paper's alternative)."""
    return modified_block_orth(W, Q, B, None, p)
