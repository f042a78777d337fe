"""Algorithm 1 (GCG) in plain FP64 -- test infrastructure only.

The iteration follows the paper's STEPs in order (Section 2, Algorithm 1, with
the implementing techniques of Sections 3.1-3.3):

* STEP 1/2  X0 (n x sizeX, sizeX = min(nev + 3 bs, n), Remark after Eq. (24))
            is B-orthonormalised by Algorithm 3; P = W = [].
* STEP 3    Rayleigh-Ritz on the unlocked block V_a = [X_a, P, W] (internal
            locking, Section 3.2): here the *full* Abar = V_a^T A V_a is formed
            explicitly and G = V_a^T B V_a is checked against I (the GPU path
            instead assembles Abar from the structure of Eq. (struct_bar_A_new)).
            The lowest sizeX - l Ritz pairs are kept.
* STEP 4    relative residuals in column order; the converged *prefix* is
            locked; blockSize = min(bs, nev - l).
* STEP 5    p~ = columns of the Ritz block for the next active block with the
            rows of the previous active block X_n zeroed (Eq. CP_tilde),
            L2-orthogonalised against the Ritz block and itself (Eq.
            Equality_Cpx); P = V_a p^.
* STEP 6    theta = largest locked eigenvalue (0 before the first lock),
            column-wise CG on (A - theta B) W = B X_n (Lambda_n - theta).
* STEP 2    W is B-orthogonalised against [X_c, X, P] and by Algorithm 3.
* Moving    (Section 3.3) a window of 3 bs X columns, P and W of bs; when
            2 bs pairs have locked inside the window, all Ritz pairs of Abar are
            taken, X = V_a [x^, p^, w^], the locked ones move to a store, the
            next (at most 3 bs) unlocked Ritz vectors form the new window and
            P = W = [] for that iteration.

Readings where the paper is silent or ambiguous:
* theta = 0 before the first lock (Remark 3.1 allows 0 <= theta);
* P is built for the *next* active block (blockSize columns), and the rows
  zeroed are those of the active block X_n that produced W in this iteration;
* p~ directions whose Gram eigenvalue after projection is <= max(1e-14 max,
  p_drop^2) are dropped (the same relative-plus-floor test as Algorithm 3's leaf);
* in moving mode the new window keeps min(sizeX, d - locked) Ritz vectors (sizeX =
  3 bs by default) and
  W is always deflated against the whole store as well;
* one iteration = one Rayleigh-Ritz solve (the initial one counts as 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .linalg import spmm, b_norms, sym_eig, residual_norms
from .cg import shifted_cg
from .orth import OrthParams, b_orthonormalize, b_orthonormalize_alg2


@dataclass
class Params:
    cg_max_iter: int = 30
    cg_rtol: float = 1e-2
    use_shift: bool = True
    max_iter: int = 1000
    p_drop: float = 1e-10
    moving: bool = False
    size_x: int | None = None
    orth: OrthParams = field(default_factory=OrthParams)
    orth_alg: int = 3            # STEP 2 by Algorithm 3 (default) or Algorithm 2
    precond: bool = False        # STEP 6 by Jacobi-preconditioned CG (oracle/cg.py)
    # optional observer called with a dict at the start of STEP 3 and at STEPs 5 and 6
    # (tests read the iteration's blocks through it, the benchmark its timing; it never
    # changes the iteration)
    trace: object = None


@dataclass
class Result:
    evals: np.ndarray
    evecs: np.ndarray
    nconv: int
    iterations: int
    converged: bool
    history: list


def p_tilde(xh: np.ndarray, c: int, bs_new: int, nb_old: int) -> np.ndarray:
    """Eq. CP_tilde: the Ritz coefficients of the next active block with the rows of
    the old active block X_n zeroed (its rows come first in V_a = [X_a, P, W])."""
    pt = np.array(xh[:, c:c + bs_new], copy=True)
    pt[:nb_old, :] = 0.0
    return pt


def _l2_orthonormal_against(pt: np.ndarray, xh: np.ndarray, drop: float) -> np.ndarray:
    """STEP 5 small dense part: orthogonalise p~ against the orthonormal x^ and itself (L2)."""
    for _ in range(2):
        for _ in range(2):
            pt = pt - xh @ (xh.T @ pt)
        if pt.shape[1] == 0:
            return pt
        lam, Q = sym_eig(pt.T @ pt)
        keep = lam > max(1e-14 * float(np.max(lam)), drop * drop)
        pt = pt @ (Q[:, keep] / np.sqrt(lam[keep])[None, :])
    return pt


def gcg(A, B, nev: int, bs: int, tol: float, X0: np.ndarray, params: Params = Params()) -> Result:
    """Smallest ``nev`` eigenpairs of A x = lambda B x by Algorithm 1.

    A: CSR symmetric; B: CSR SPD or None (identity); X0: n x sizeX initial block.
    """
    p = params
    n = A.shape[0]
    if p.size_x is not None:
        size_x = p.size_x
    elif p.moving:
        size_x = min(3 * bs, n)
    else:
        size_x = min(nev + 3 * bs, n)
    if X0.shape != (n, size_x):
        raise ValueError(f"X0 must be {n} x {size_x}")

    borth = b_orthonormalize if p.orth_alg == 3 else b_orthonormalize_alg2
    # ---- STEP 1/2: orthonormalise the initial block (Algorithm 3, or Algorithm 2)
    X, _ = borth(np.array(X0, dtype=np.float64), None, B, p.orth)
    if X.shape[1] != size_x:
        raise ValueError("initial block is rank deficient")
    lam = np.zeros(size_x)
    store = np.zeros((n, 0))
    store_lam = np.zeros(0)
    lw = 0                       # locked columns inside the window X
    P = np.zeros((n, 0))
    W = np.zeros((n, 0))
    nb_old = 0                   # size of the active block that produced W
    history = []
    it = 0
    converged = False
    while True:
        it += 1
        if p.trace is not None:
            p.trace(dict(step=3, it=it))
        # ---- STEP 3: Rayleigh-Ritz on V_a = [X_a, P, W] with an explicit V^T A V
        Va = np.hstack([X[:, lw:], P, W])
        AVa = spmm(A, Va)
        BVa = spmm(B, Va)
        Abar = Va.T @ AVa
        G = Va.T @ BVa
        orth_err = float(np.max(np.abs(G - np.eye(G.shape[0]))))
        theta_all, Q = sym_eig(Abar)
        d = Va.shape[1]
        kx = X.shape[1] - lw
        # ---- STEP 4: convergence of the new unlocked Ritz pairs, prefix locking
        Xa_new = Va @ Q[:, :kx]
        res = residual_norms(A, B, Xa_new, theta_all[:kx])
        c = 0
        while c < kx and res[c] < tol:
            c += 1
        l_total = store.shape[1] + lw + c
        # Section 3.3 moves the window once 2 blockSize new pairs have converged.  It
        # is also moved when every unlocked vector of X has converged (the paper does
        # not treat this case): X would otherwise keep no vector to iterate on
        move = p.moving and l_total < nev and ((lw + c) >= 2 * bs or c == kx)
        history.append(dict(it=it, nconv=min(l_total, nev), d=d, orth_err=orth_err,
                            res_first=float(res[c]) if c < kx else 0.0,
                            nP=P.shape[1], nW=W.shape[1], kx=kx, c=c, lw=lw, move=move))
        if move:
            # ---- moving mechanism: all Ritz vectors of Abar, flush the locked ones
            Xall = Va @ Q
            store = np.hstack([store, X[:, :lw], Xall[:, :c]])
            store_lam = np.concatenate([store_lam, lam[:lw], theta_all[:c]])
            keep = min(size_x, d - c)
            X = Xall[:, c:c + keep]
            lam = theta_all[c:c + keep].copy()
            lw = 0
            P = np.zeros((n, 0))
        else:
            X = np.hstack([X[:, :lw], Xa_new])
            lam = np.concatenate([lam[:lw], theta_all[:kx]])
            lw += c
        l_total = store.shape[1] + lw
        if l_total >= nev:
            converged = True
            break
        if X.shape[1] - lw == 0:
            raise RuntimeError("the search window holds no unlocked vector")
        if it >= p.max_iter:
            break
        bs_new = min(bs, nev - l_total, X.shape[1] - lw)
        # ---- STEP 5: P from the Ritz block (skipped right after a move)
        if not move:
            if nb_old == 0 or bs_new <= 0:
                P = np.zeros((n, 0))
            else:
                xh = Q[:, :kx]
                ph = _l2_orthonormal_against(p_tilde(xh, c, bs_new, nb_old), xh, p.p_drop)
                P = Va @ ph
                if p.trace is not None:
                    p.trace(dict(step=5, it=it, Xnew=Xa_new, c=c, bs_new=bs_new, P=P))
        # ---- STEP 6: shifted CG from the active block
        locked_lam = np.concatenate([store_lam, lam[:lw]])
        theta = float(np.max(locked_lam)) if (p.use_shift and locked_lam.size) else 0.0
        Xn = X[:, lw:lw + bs_new]
        if p.trace is not None:
            p.trace(dict(step=6, it=it, Xn=Xn))
        Wt, cg_it, _ = shifted_cg(A, B, theta, Xn, lam[lw:lw + bs_new], p.cg_max_iter, p.cg_rtol,
                                  precond=p.precond)
        history[-1].update(theta=theta, cg_iters=int(cg_it.max()) if cg_it.size else 0)
        # ---- STEP 2: B-orthogonalise W against [X_c (store), X, P], then Algorithm 3
        Q0 = np.hstack([store, X, P])
        W, _ = borth(Wt, Q0, B, p.orth)
        nb_old = bs_new

    allX = np.hstack([store, X[:, :lw]])
    allL = np.concatenate([store_lam, lam[:lw]])
    order = np.argsort(allL, kind="stable")
    k = min(nev, allL.size)
    return Result(allL[order][:k], allX[:, order][:, :k], int(allL.size), it, converged, history)
