"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form
printed in the paper (Remark 3.1), closed-form spectra of the discretisations,
textbook invariants (CG residual orthogonality, V^T B V = I, Eq. Equality_xx /
Equality_xp / Equality_Cpx), brute-force dense solves on tiny pencils, and
homogeneity/finite-difference identities for gradients.  A few tests plant a
mistake in the oracle (on the CPU) and check that a pin catches it.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

import workloads as W
from oracle import linalg as L
from oracle import cg as CG
from oracle import orth as O
from oracle import gcg as G
from oracle import grad as GR

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- SpMM
def test_spmm_on_sine_modes_gives_eigenvalues():
    N = 11
    p = W.fd2d(N)
    h = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    modes = [(1, 1), (2, 3), (5, 4)]
    X = np.stack([np.outer(np.sin(a * np.pi * i * h), np.sin(b * np.pi * i * h)).ravel()
                  for a, b in modes], axis=1)
    lam = np.array([(4 / h ** 2) * (np.sin(a * np.pi * h / 2) ** 2 + np.sin(b * np.pi * h / 2) ** 2)
                    for a, b in modes])
    Y = L.spmm(p.A, X)
    assert np.abs(Y - X * lam).max() <= 1e-11 * lam.max()
    assert np.array_equal(L.spmm(None, X), X)


def test_residual_norm_is_zero_for_exact_pairs():
    p = W.q1_kron(5)
    ev, V = sl.eigh(p.A.toarray(), p.B.toarray())
    r = L.residual_norms(p.A, p.B, V[:, :6], ev[:6])
    assert r.max() < 1e-12
    r2 = L.residual_norms(p.A, p.B, V[:, :6], ev[:6] * (1 + 1e-6))
    # a relative eigenvalue error dl gives exactly dl ||B x||_2 / ||x||_B
    BV = p.B @ V[:, :6]
    expect = 1e-6 * np.linalg.norm(BV, axis=0) / np.sqrt(np.einsum("ij,ij->j", V[:, :6], BV))
    assert np.allclose(r2, expect, rtol=1e-5)


# ---------------------------------------------------------------- CG (STEP 6)
def _remark_cases():
    return json.load(open(os.path.join(GOLD, "remark31.json")))["cases"]


@pytest.mark.parametrize("case", _remark_cases())
def test_cg_one_step_matches_remark_3_1(case):
    l1, l2, l3, a2, a3, th = (case[k] for k in ("l1", "l2", "l3", "a2", "a3", "theta"))
    import scipy.sparse as sp
    A = sp.csr_matrix(np.diag([l1, l2, l3]))
    x0 = np.array([0.0, a2, a3])
    lt = x0 @ (A @ x0) / (x0 @ x0)
    rhs = ((lt - th) * x0)[:, None]
    x1, it, _ = CG.shifted_cg(A, None, th, x0[:, None], np.array([lt]), max_iter=1, rtol=0.0,
                              rhs=rhs)
    coef = (a2 ** 2 + a3 ** 2) / (a3 ** 2 * (l2 - th) + a2 ** 2 * (l3 - th))
    expect = coef * np.array([0.0, (l3 - th) * a2, (l2 - th) * a3])
    # with l2 == l3 the start is already an eigenvector: r0 = 0 and CG takes no step
    assert it[0] == (0 if l2 == l3 else 1)
    assert np.abs(x1[:, 0] - expect).max() <= 1e-14 * np.abs(expect).max()


def test_cg_solves_spd_system_and_residuals_are_orthogonal():
    A = W.random_sparse_spd(60, 0.1, 3)
    rng = np.random.default_rng(0)
    b = rng.standard_normal((60, 2))
    x0 = rng.standard_normal((60, 2))
    # run k = 1..8 steps and record residuals to test r_k^T r_j = 0
    res = []
    for k in range(1, 9):
        x, _, _ = CG.shifted_cg(A, None, 0.0, x0, np.zeros(2), max_iter=k, rtol=0.0, rhs=b)
        res.append(b - A @ x)
    R = np.stack([r[:, 0] for r in res], axis=1)
    Rn = R / np.linalg.norm(R, axis=0)
    offd = Rn.T @ Rn - np.eye(R.shape[1])
    assert np.abs(offd).max() < 1e-8
    x, it, broke = CG.shifted_cg(A, None, 0.0, x0, np.zeros(2), max_iter=200, rtol=1e-13, rhs=b)
    xs = np.linalg.solve(A.toarray(), b)
    assert np.abs(x - xs).max() <= 1e-11 * np.abs(xs).max()
    assert not broke.any() and it.max() < 200


def test_cg_stopping_rule_and_breakdown():
    A = W.random_sparse_spd(80, 0.08, 4)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((80, 3))
    lam = np.array([1.0, 2.0, 3.0])
    W_, it, broke = CG.shifted_cg(A, None, 0.5, X, lam, max_iter=30, rtol=1e-2)
    S = CG.shifted_matrix(A, None, 0.5)
    b = X * (lam - 0.5)
    r0 = np.linalg.norm(b - S @ X, axis=0)
    r = np.linalg.norm(b - S @ W_, axis=0)
    for j in range(3):
        assert it[j] == 30 or r[j] <= 1e-2 * r0[j] * (1 + 1e-12)
    # an indefinite shift breaks down: p^T S p <= 0 for the first direction
    ev = np.linalg.eigvalsh(A.toarray())
    x = np.linalg.eigh(A.toarray())[1][:, :1]
    _, it2, broke2 = CG.shifted_cg(A, None, 0.5 * (ev[0] + ev[1]), x + 0.0, np.array([0.0]),
                                   max_iter=30, rtol=0.0)
    assert broke2[0] and it2[0] == 0


def _pcg_residuals(S, b, steps):
    """Residuals r_j = b - S x_j of Jacobi-preconditioned CG after j = 0..steps steps."""
    n = S.shape[0]
    out = []
    for j in range(steps + 1):
        x, it, _ = CG.shifted_cg(S, None, 0.0, np.zeros((n, 1)), np.zeros(1), max_iter=j,
                                 rtol=0.0, rhs=b[:, None], precond=True)
        out.append(b - S @ x[:, 0])
    return out


def test_pcg_residuals_are_m_orthogonal():
    """Preconditioned CG: r_i^T M^-1 r_j = 0 for i != j (textbook property), on the
    lognormal FD operator whose diagonal varies over orders of magnitude."""
    p = W.make_config("fd3d_128", N=8, seed=2)
    S = p.A
    b = np.random.default_rng(3).standard_normal(S.shape[0])
    R = np.column_stack(_pcg_residuals(S, b, 8))
    minv = CG.jacobi_inverse(S)
    G = R.T @ (R * minv[:, None])
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 1e-9 * np.sqrt(np.outer(np.diag(G), np.diag(G))).max()


def test_pcg_diagonal_system_in_one_step():
    """A diagonal S is its own Jacobi preconditioner: one step solves it exactly."""
    d = np.linspace(0.5, 300.0, 40)
    S = sp.diags(d).tocsr()
    b = np.random.default_rng(4).standard_normal(40)
    x, it, _ = CG.shifted_cg(S, None, 0.0, np.zeros((40, 1)), np.zeros(1), max_iter=1,
                             rtol=0.0, rhs=b[:, None], precond=True)
    assert np.abs(x[:, 0] - b / d).max() <= 1e-14 * np.abs(b / d).max()


def test_pcg_fewer_steps_on_high_contrast_operator():
    p = W.make_config("fd3d_128", N=12, seed=1)
    S = p.A
    b = np.random.default_rng(5).standard_normal((S.shape[0], 2))
    _, it_cg, _ = CG.shifted_cg(S, None, 0.0, np.zeros_like(b), np.zeros(2), max_iter=500,
                                rtol=1e-8, rhs=b)
    _, it_pcg, _ = CG.shifted_cg(S, None, 0.0, np.zeros_like(b), np.zeros(2), max_iter=500,
                                 rtol=1e-8, rhs=b, precond=True)
    assert it_pcg.max() < 0.7 * it_cg.max()


def test_gcg_with_jacobi_pcg_closed_form():
    p = W.make_config("q1_64", N=7)
    nev, bs = 12, 3
    r = G.gcg(p.A, p.B, nev, bs, 1e-8, W.initial_block(p.n, nev + 3 * bs, 1),
              G.Params(precond=True))
    exact = W.q1_eigs(7, nev)
    assert r.converged
    assert np.abs(r.evals - exact).max() <= 1e-8 * exact[0]


def test_planted_pcg_unpreconditioned_beta_is_caught(monkeypatch):
    # beta from r^T r instead of r^T M^-1 r breaks the M^-1-orthogonality of residuals
    orig = CG.shifted_cg

    def wrong(A, B, theta, X, lam, max_iter=30, rtol=1e-2, rhs=None, precond=False):
        n, k = X.shape
        S = CG.shifted_matrix(A, B, theta)
        minv = CG.jacobi_inverse(S)[:, None]
        x = X.copy()
        r = rhs - S @ x
        z = r * minv
        p_ = z.copy()
        rr = np.einsum("ij,ij->j", r, r)
        rz = np.einsum("ij,ij->j", r, z)
        for _ in range(max_iter):
            q = S @ p_
            alpha = rz / np.einsum("ij,ij->j", p_, q)
            x += p_ * alpha
            r -= q * alpha
            z = r * minv
            rr_new = np.einsum("ij,ij->j", r, r)
            p_ = z + p_ * (rr_new / rr)
            rr = rr_new
            rz = np.einsum("ij,ij->j", r, z)
        return x, np.full(k, max_iter), np.zeros(k, dtype=bool)

    monkeypatch.setattr(CG, "shifted_cg", wrong)
    with pytest.raises(AssertionError):
        test_pcg_residuals_are_m_orthogonal()


# ---------------------------------------------------------------- Algorithm 3 / 2 (STEP 2)
def _pencil_small():
    p = W.make_config("q1grad_48", N=6, seed=3)
    return p.A, p.B


def _proj(X, BX):
    return X @ BX.T          # B-orthogonal projector expressed as X X^T B (transposed form)


@pytest.mark.parametrize("m", [1, 5, 16, 17, 20, 37])
def test_recursive_orth_svd_orthonormal_and_same_span(m):
    A, B = _pencil_small()
    rng = np.random.default_rng(m)
    X = rng.standard_normal((B.shape[0], m))
    Y, BY = O.b_orthonormalize(X, None, B)
    assert Y.shape[1] == m
    assert np.abs(Y.T @ (B @ Y) - np.eye(m)).max() < 1e-13
    assert np.abs(BY - B @ Y).max() < 1e-12 * np.abs(BY).max()
    # same span: X is reproduced by its B-projection onto span(Y)
    Xp = Y @ (BY.T @ X)
    assert np.abs(Xp - X).max() < 1e-11 * np.abs(X).max()


def test_orth_drops_dependent_columns_and_deflates():
    A, B = _pencil_small()
    rng = np.random.default_rng(7)
    Q0, _ = O.b_orthonormalize(rng.standard_normal((B.shape[0], 6)), None, B)
    X = rng.standard_normal((B.shape[0], 5))
    X[:, 3] = 2.0 * X[:, 1] - X[:, 0]             # dependent inside the block
    X[:, 4] = Q0 @ rng.standard_normal(6)           # inside span(Q0)
    Y, BY = O.b_orthonormalize(X, Q0, B)
    assert Y.shape[1] == 3
    assert np.abs(Q0.T @ BY).max() < 1e-13
    assert np.abs(Y.T @ BY - np.eye(3)).max() < 1e-13


def test_deflation_keeps_small_new_directions():
    """A correction that differs from span(Q) by 1e-11 (a pair near its tolerance)
    keeps its new direction -- exactly that direction, B-normalised -- while a
    column inside span(Q) up to rounding is dropped."""
    A, B = _pencil_small()
    rng = np.random.default_rng(11)
    n = B.shape[0]
    Q, _ = O.b_orthonormalize(rng.standard_normal((n, 4)), None, B)
    z = rng.standard_normal(n)
    z -= Q @ (Q.T @ (B @ z))
    z /= np.sqrt(z @ (B @ z))                       # B-unit, B-orthogonal to Q
    w_small = Q[:, 0] + 1e-11 * z                   # new direction of relative size 1e-11
    w_inside = Q @ rng.standard_normal(4)           # no new direction at all
    Wd, BWd = O.deflate_against(np.column_stack([w_small, w_inside]), Q, B)
    assert Wd.shape[1] == 1
    cos = abs(Wd[:, 0] @ (B @ z)) / np.sqrt(Wd[:, 0] @ BWd[:, 0])
    assert cos > 1 - 1e-6


def test_modified_block_orth_alg2():
    A, B = _pencil_small()
    rng = np.random.default_rng(8)
    X = rng.standard_normal((B.shape[0], 24))
    Y, BY = O.modified_block_orth(X, None, B)
    assert Y.shape[1] == 24
    assert np.abs(Y.T @ BY - np.eye(24)).max() < 1e-13
    assert np.abs(Y @ (BY.T @ X) - X).max() < 1e-11 * np.abs(X).max()


@pytest.mark.parametrize("withB", [False, True])
def test_alg2_equals_cholesky_qr(withB):
    """Block modified Gram-Schmidt takes each column against all earlier ones in
    order, so without drops it gives the B-QR factor X R^-1 with R the Cholesky factor
    of X^T B X (positive diagonal) -- a textbook routine, whatever the block size."""
    A, B = _pencil_small()
    B = B if withB else None
    rng = np.random.default_rng(11)
    n = A.shape[0]
    X = rng.standard_normal((n, 20)) @ np.diag(np.logspace(0, -3, 20))
    BX = X if B is None else B @ X
    s = np.sqrt(np.einsum("ij,ij->j", X, BX))
    Xs = X / s                           # Algorithm 2 starts from unit B-norm columns
    R = np.linalg.cholesky(Xs.T @ (Xs if B is None else B @ Xs)).T
    Yref = np.linalg.solve(R.T, Xs.T).T
    for b in (1, 5, 7, 20):
        Y, BY = O.modified_block_orth(X, None, B, b)
        assert Y.shape[1] == 20
        assert np.abs(Y - Yref).max() < 1e-9 * np.abs(Yref).max()


def test_alg2_drops_dependent_columns():
    A, B = _pencil_small()
    rng = np.random.default_rng(12)
    n = A.shape[0]
    Q, _ = O.b_orthonormalize(rng.standard_normal((n, 4)), None, B)
    X = rng.standard_normal((n, 12))
    X[:, 5] = X[:, 1] + X[:, 2]                # inside the block's own span
    X[:, 9] = Q @ rng.standard_normal(4)       # inside span(Q)
    Y, BY = O.modified_block_orth(X, Q, B, 3)
    assert Y.shape[1] == 10
    assert np.abs(Y.T @ BY - np.eye(10)).max() < 1e-12
    assert np.abs(Q.T @ BY).max() < 1e-12
    # span(Y) + span(Q) holds every input column
    QY = np.hstack([Q, Y])
    res = X - QY @ (np.hstack([B @ Q, BY]).T @ X)
    assert np.abs(res).max() < 1e-10 * np.abs(X).max()


def test_gcg_with_alg2_closed_form():
    p = W.fd2d(16)
    nev, bs = 12, 3
    r = G.gcg(p.A, None, nev, bs, 1e-8, W.initial_block(p.n, nev + 3 * bs, 2),
              G.Params(orth_alg=2))
    exact = W.fd2d_eigs(16, nev)
    assert r.converged
    assert np.abs(r.evals - exact).max() <= 1e-8 * exact[0]


# ---------------------------------------------------------------- full GCG (Algorithm 1)
def test_gcg_fd2d_closed_form():
    p = W.fd2d(20)
    nev, bs = 20, 10
    X0 = W.initial_block(p.n, nev + 3 * bs, 0)
    r = G.gcg(p.A, None, nev, bs, 1e-8, X0)
    ex = W.fd2d_eigs(20, nev)
    assert r.converged
    assert np.abs(r.evals - ex).max() <= 1e-8 * ex.min()
    assert L.residual_norms(p.A, None, r.evecs, r.evals).max() < 1e-8
    assert np.abs(r.evecs.T @ r.evecs - np.eye(nev)).max() < 1e-12


def test_gcg_q1_closed_form_generalized():
    p = W.q1_kron(8)
    nev, bs = 24, 5
    X0 = W.initial_block(p.n, nev + 3 * bs, 1)
    r = G.gcg(p.A, p.B, nev, bs, 1e-8, X0)
    ex = W.q1_eigs(8, nev)
    assert r.converged
    assert np.abs(r.evals - ex).max() <= 1e-8 * ex.min()
    assert np.abs(r.evecs.T @ (p.B @ r.evecs) - np.eye(nev)).max() < 1e-12


@pytest.mark.parametrize("name,N,nev,bs", [("fd3d_128", 8, 12, 3), ("q1_160", 5, 15, 3),
                                           ("q1grad_48", 6, 10, 2)])
def test_gcg_brute_force_on_variable_coefficient(name, N, nev, bs):
    p = W.make_config(name, N=N, seed=5)
    Bd = p.B.toarray() if p.B is not None else None
    ev, V = sl.eigh(p.A.toarray(), Bd)
    X0 = W.initial_block(p.n, nev + 3 * bs, 2)
    r = G.gcg(p.A, p.B, nev, bs, 1e-9, X0)
    assert r.converged
    assert np.abs(r.evals - ev[:nev]).max() <= 1e-8 * ev[0]
    # eigenvectors: subspace of the computed block equals the exact one (gap-separated cut)
    Bm = Bd if Bd is not None else np.eye(p.n)
    s = np.linalg.svd(V[:, :nev].T @ Bm @ r.evecs, compute_uv=False)
    assert s.min() > 1 - 1e-10


def test_gcg_moving_matches_plain():
    p = W.fd2d(20)
    nev, bs = 30, 4
    r1 = G.gcg(p.A, None, nev, bs, 1e-8, W.initial_block(p.n, nev + 3 * bs, 0))
    r2 = G.gcg(p.A, None, nev, bs, 1e-8, W.initial_block(p.n, 3 * bs, 0), G.Params(moving=True))
    assert r1.converged and r2.converged
    ex = W.fd2d_eigs(20, nev)
    assert np.abs(r1.evals - ex).max() <= 1e-8 * ex[0]
    assert np.abs(r2.evals - ex).max() <= 1e-8 * ex[0]
    assert max(h["d"] for h in r2.history) <= 5 * bs


@pytest.mark.parametrize("N,nev,bs,seed", [(18, 30, 4, 1), (16, 24, 3, 9), (14, 20, 2, 4)])
def test_gcg_moving_window_exhaustion(N, nev, bs, seed):
    """Section 3.3: on these starts every unlocked vector of the window converges
    before 2 blockSize new pairs are locked.  The window is then moved (P and W fold
    into X) instead of being left empty, and the run reaches the closed-form spectrum."""
    p = W.fd2d(N)
    r = G.gcg(p.A, None, nev, bs, 1e-8, W.initial_block(p.n, 3 * bs, seed), G.Params(moving=True))
    assert r.converged
    ex = W.fd2d_eigs(N, nev)
    assert np.abs(r.evals - ex).max() <= 1e-8 * ex[0]
    early = [h for h in r.history if h["move"] and h["c"] == h["kx"] and h["lw"] + h["c"] < 2 * bs]
    assert early, "the case no longer exercises a move on an exhausted window"
    assert max(h["d"] for h in r.history) <= 5 * bs


def test_gcg_shift_reduces_iterations():
    p = W.fd2d(24)
    nev, bs = 30, 3
    X0 = W.initial_block(p.n, nev + 3 * bs, 4)
    r1 = G.gcg(p.A, None, nev, bs, 1e-8, X0, G.Params(cg_max_iter=10))
    r0 = G.gcg(p.A, None, nev, bs, 1e-8, X0, G.Params(cg_max_iter=10, use_shift=False))
    assert r1.converged and r0.converged
    assert r1.iterations < r0.iterations


def test_gcg_invariants_each_iteration():
    # V^T B V = I at every Rayleigh-Ritz (checked inside the oracle and recorded)
    p = W.q1_kron(7)
    r = G.gcg(p.A, p.B, 12, 3, 1e-8, W.initial_block(p.n, 21, 9))
    assert max(h["orth_err"] for h in r.history) < 1e-12
    assert all(h["nconv"] <= 12 for h in r.history)
    nc = [h["nconv"] for h in r.history]
    assert nc == sorted(nc)


# ---------------------------------------------------------------- gradients
def _grad_setup(N=4, seed=2, k=3):
    p = W.make_config("q1grad_48", N=N, seed=seed)
    ev, V = sl.eigh(p.A.toarray(), p.B.toarray())
    return p, ev, V, k


def test_grad_eigenvalue_euler_and_fd():
    p, ev, V, k = _grad_setup()
    N = 4
    c = p.meta["c"].ravel()
    for i in range(k):
        g = GR.cell_bilinear(N, V[:, i], V[:, i])
        assert abs((g * c).sum() - ev[i]) <= 1e-12 * ev[i]
    e = 17
    d = 1e-5 * c[e]
    cp, cm = c.copy(), c.copy()
    cp[e] += d
    cm[e] -= d
    Bd = p.B.toarray()
    lp = sl.eigh(W.q1_var(N, cp).A.toarray(), Bd, eigvals_only=True)[0]
    lm = sl.eigh(W.q1_var(N, cm).A.toarray(), Bd, eigvals_only=True)[0]
    g = GR.cell_bilinear(N, V[:, 0], V[:, 0])
    assert abs((lp - lm) / (2 * d) - g[e]) <= 1e-6 * abs(g).max()


def test_grad_adjoint_matches_full_spectrum_and_fd():
    p, ev, V, k = _grad_setup()
    N = 4
    c = p.meta["c"].ravel()
    rng = np.random.default_rng(3)
    S = (rng.uniform(size=p.n) < 0.3).astype(float)
    Bd = p.B.toarray()
    BS = (S[:, None] * Bd) * S[None, :]
    wts = rng.uniform(size=k)
    # L = sum_i w_i x_i^T B_S x_i; dL/dx_i = 2 w_i B_S x_i
    Gx = np.stack([2 * wts[i] * BS @ V[:, i] for i in range(k)], axis=1)
    for i in range(k):
        mu = GR.adjoint(p.A, p.B, ev[:k], V[:, :k], i, Gx[:, i])
        mu_full = sum(V[:, j] * (V[:, j] @ Gx[:, i]) / (ev[j] - ev[i])
                      for j in range(p.n) if j != i)
        assert np.abs(mu - mu_full).max() <= 1e-9 * np.abs(mu_full).max()
    g = GR.loss_grad_cells(N, p.A, p.B, ev[:k], V[:, :k], np.zeros(k), Gx)
    assert abs((g * c).sum()) <= 1e-9 * np.abs(g * c).sum()      # scale invariance of x_i

    def loss(cc):
        e2, V2 = sl.eigh(W.q1_var(N, cc).A.toarray(), Bd)
        return sum(wts[i] * V2[:, i] @ BS @ V2[:, i] for i in range(k))

    for e in (3, 40):
        d = 1e-5 * c[e]
        cp, cm = c.copy(), c.copy()
        cp[e] += d
        cm[e] -= d
        fd = (loss(cp) - loss(cm)) / (2 * d)
        assert abs(fd - g[e]) <= 1e-5 * abs(g).max()


def test_grad_nonzero_form_chains_to_cells():
    p, ev, V, k = _grad_setup()
    N = 4
    w = np.array([1.0, 0.5, 0.25])
    gnz = GR.loss_grad_nonzeros(p.A, ev[:k], V[:, :k], w, None)
    # chain rule through dA_pq/dc_e = Khat[a, b] equals the per-cell formula
    gcell = sum(w[i] * GR.cell_bilinear(N, V[:, i], V[:, i]) for i in range(k))
    c = p.meta["c"].ravel()
    dc = np.random.default_rng(0).standard_normal(c.size)
    dA = W.q1_var(N, dc).A              # A is linear in c: dA = A(dc)
    assert abs(gnz @ dA.data - gcell @ dc) <= 1e-12 * np.abs(gcell).sum()


# ---------------------------------------------------------------- planted mistakes
def test_planted_cg_sign_error_is_caught(monkeypatch):
    case = _remark_cases()[1]
    orig = CG.shifted_cg

    def wrong(A, B, theta, *a, **k):           # sign error on the shift
        return orig(A, B, -theta, *a, **k)

    monkeypatch.setattr(CG, "shifted_cg", wrong)
    with pytest.raises(AssertionError):
        test_cg_one_step_matches_remark_3_1(case)


def test_planted_orth_missing_deflation_is_caught(monkeypatch):
    def no_defl(W_, Q, B, p=O.OrthParams()):
        BW = L.spmm(B, W_)
        return O.normalize_cols(W_, BW)

    monkeypatch.setattr(O, "deflate_against", no_defl)
    with pytest.raises(AssertionError):
        test_orth_drops_dependent_columns_and_deflates()


def test_planted_missing_p_projection_is_caught(monkeypatch):
    # without the L2 orthogonalisation of p~ against x^ (Eq. Equality_Cpx) P stays
    # coupled to X and the basis V_a loses its B-orthonormality
    def skip_projection(pt, xh, drop):
        lam, Q = L.sym_eig(pt.T @ pt)
        keep = lam > drop * drop
        return pt @ (Q[:, keep] / np.sqrt(lam[keep])[None, :])

    monkeypatch.setattr(G, "_l2_orthonormal_against", skip_projection)
    p = W.q1_kron(6)
    r = G.gcg(p.A, p.B, 8, 2, 1e-8, W.initial_block(p.n, 14, 0), G.Params(max_iter=6))
    assert max(h["orth_err"] for h in r.history) > 1e-6


# ---------------------------------------------------------------- STEP 5 (P)
def _b_basis(Y, B):
    """A B-orthonormal basis of span(Y) (test-side, dense)."""
    BY = Y if B is None else B @ Y
    lam, Q = np.linalg.eigh(Y.T @ BY)
    keep = lam > 1e-20 * max(lam.max(), 1e-300)
    return Y @ (Q[:, keep] / np.sqrt(lam[keep]))


def _step5_pin(pencil, nev, bs, seed, max_iter, moving=False):
    """P^new of the oracle against the paper's own definition before Eq. CP_tilde:
    P~ = V x^_n - X_n (X_n^T B V x^_n), with X_n the block that produced W (recorded
    at STEP 6 of the previous iteration) and V x^_n the new Ritz vectors of the next
    active block; P^new must span P~ B-orthogonalised against X^new, and satisfy
    (X^new)^T B P^new = O, (P^new)^T B P^new = I (the identities after Eq. Equality_Cpx)."""
    events = []
    size_x = 3 * bs if moving else nev + 3 * bs
    X0 = W.initial_block(pencil.n, size_x, seed)
    G.gcg(pencil.A, pencil.B, nev, bs, 1e-8, X0,
          G.Params(max_iter=max_iter, moving=moving, trace=events.append))
    B = pencil.B
    Bm = (lambda Y: Y) if B is None else (lambda Y: B @ Y)
    checked = 0
    xn_prev = None
    for e in events:
        if e["step"] == 6:
            xn_prev = e["Xn"]
            continue
        if e["step"] != 5:
            continue
        Xnew, c, b, P = e["Xnew"], e["c"], e["bs_new"], e["P"]
        Vxn = Xnew[:, c:c + b]
        Pt = Vxn - xn_prev @ (xn_prev.T @ Bm(Vxn))
        for _ in range(2):
            Pt = Pt - Xnew @ (Bm(Xnew).T @ Pt)
        # P~ is a difference of nearly equal blocks once X_n has nearly converged; its
        # direction is then fixed only to eps / sigma_min(P~), so such steps are skipped
        if np.linalg.eigvalsh(Pt.T @ Bm(Pt)).min() < 1e-12:
            continue
        Qt = _b_basis(Pt, B)
        BP = Bm(P)
        assert P.shape[1] == Qt.shape[1] == b
        assert np.abs(P.T @ BP - np.eye(b)).max() < 1e-10
        assert np.abs(Xnew.T @ BP).max() < 1e-10
        # span(P^new) = span(P~ projected): the part of P outside span(Qt) vanishes
        outside = P - Qt @ (Qt.T @ BP)
        assert np.sqrt(np.einsum("ij,ij->j", outside, Bm(outside))).max() < 1e-8
        checked += 1
    assert checked >= 3
    return checked


@pytest.mark.parametrize("name,moving", [("q1var", False), ("fd2d", False), ("fd2d", True)])
def test_step5_p_spans_paper_definition(name, moving):
    if name == "q1var":
        p = W.q1_var(6, W.lognormal_cells((7, 7, 7), 1.0, 3))
        _step5_pin(p, 8, 2, 0, 8)
    else:
        p = W.fd2d(12)
        _step5_pin(p, 12, 2, 1, 12, moving=moving)


def test_planted_wrong_p_rows_is_caught(monkeypatch):
    # Eq. CP_tilde zeroes the rows of the old active block X_n; zeroing the next
    # nb_old rows (those of X_n~) instead must fail the STEP 5 pin
    def wrong_rows(xh, c, bs_new, nb_old):
        pt = np.array(xh[:, c:c + bs_new], copy=True)
        pt[nb_old:2 * nb_old, :] = 0.0
        return pt

    monkeypatch.setattr(G, "p_tilde", wrong_rows)
    p = W.q1_var(6, W.lognormal_cells((7, 7, 7), 1.0, 3))
    with pytest.raises(AssertionError):
        _step5_pin(p, 8, 2, 0, 8)


def test_planted_no_p_is_caught(monkeypatch):
    # P never formed (p~ empty): the pin sees a P of the wrong width
    monkeypatch.setattr(G, "p_tilde", lambda xh, c, bs_new, nb_old: xh[:, :0].copy())
    p = W.q1_var(6, W.lognormal_cells((7, 7, 7), 1.0, 3))
    with pytest.raises(AssertionError):
        _step5_pin(p, 8, 2, 0, 8)
