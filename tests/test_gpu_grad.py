"""Differentiation of the eigensolver (not in the paper): adjoint gradients vs the oracle.

L = sum_i lambda_i + sum_i w_i x_i^T B_S x_i on the Q1 pencil with cell coefficients c.
The GPU gradient goes c -> A(c).data (library SpMM with the cell Jacobian) -> gcge_solve
-> torch loss -> gcge_eig_grad (adjoint kernel) -> J^T (library SpMM).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import gcg as G
from oracle import grad as GR

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    import paper_2111_06552_gb300 as gg
    assert torch.cuda.is_available()
    gg.lib()
    return gg


def _gpu_grad(g, N, setup, nev, bs, tol=1e-10, use_vec=True, c=None):
    import torch
    c = setup["c"] if c is None else c
    p = W.q1_var(N, c)
    J = W.q1_cell_jacobian(N, p.A)
    cmap = g.CellMap(J)
    rp = torch.tensor(p.A.indptr.astype(np.int32), device="cuda")
    ci = torch.tensor(p.A.indices.astype(np.int32), device="cuda")
    ct = torch.tensor(c.ravel(), dtype=torch.float64, device="cuda", requires_grad=True)
    a = g.cells_to_values(ct, cmap)
    ev, X = g.EigGCG.apply(a, (rp, ci), p.B, nev, bs, tol, 1e-12, {"seed": 0})
    loss = ev.sum()
    if use_vec:
        Sm = sp.diags(setup["S"])
        BS = (Sm @ p.B @ Sm).tocsr().tocoo()
        BSt = torch.sparse_coo_tensor(np.vstack([BS.row, BS.col]), BS.data, BS.shape,
                                      device="cuda").coalesce()
        w = torch.tensor(setup["w"][:nev], device="cuda")
        loss = loss + (w * (X * torch.sparse.mm(BSt, X)).sum(0)).sum()
    loss.backward()
    return ct.grad.cpu().numpy(), ev.detach().cpu().numpy(), X.detach().cpu().numpy(), p


def test_gradient_matches_oracle_small(g):
    N, nev, bs = 6, 6, 2
    st = W.q1grad_setup(N, seed=3, nev=nev, sub=3)
    grad, ev, X, p = _gpu_grad(g, N, st, nev, bs)
    # oracle: eigenpairs by the FP64 GCG oracle, gradient by its adjoint formulas
    r = G.gcg(p.A, p.B, nev, bs, 1e-10, W.initial_block(p.n, nev + 3 * bs, 0))
    Sm = sp.diags(st["S"])
    BS = (Sm @ p.B @ Sm).tocsr()
    Gx = np.stack([2 * st["w"][i] * (BS @ r.evecs[:, i]) for i in range(nev)], axis=1)
    ref = GR.loss_grad_cells(N, p.A, p.B, r.evals, r.evecs, np.ones(nev), Gx, tol=1e-13)
    assert np.abs(ev - r.evals).max() <= 1e-9 * r.evals.max()
    assert np.abs(grad - ref).max() <= 1e-6 * np.abs(ref).max()


def test_gradient_homogeneity(g):
    N, nev, bs = 7, 6, 2
    st = W.q1grad_setup(N, seed=5, nev=nev, sub=4)
    c = st["c"].ravel()
    gl, ev, X, p = _gpu_grad(g, N, st, nev, bs, use_vec=False)
    # eigenvalues are homogeneous of degree 1 in c (B fixed): sum_e c_e dlam/dc_e = sum lam
    assert abs((gl * c).sum() - ev.sum()) <= 1e-9 * ev.sum()
    gt, _, _, _ = _gpu_grad(g, N, st, nev, bs, use_vec=True)
    gv = gt - gl          # eigenvector part alone: x_i are invariant to scaling c
    assert abs((gv * c).sum()) <= 1e-7 * np.abs(gv * c).sum()


def _loss_fd(g, N, st, c, nev, bs, tol):
    """L = sum lambda_i + sum_i w_i x_i^T B_S x_i from a fresh GPU solve (no gradient)."""
    p = W.q1_var(N, c)
    s = g.Solver(p.A, p.B, nev, bs, tol, seed=0)
    ev, X = s.solve()
    s.close()
    X = np.array(X)
    Sm = sp.diags(st["S"])
    BSX = Sm @ (p.B @ (Sm @ X))
    return ev.sum() + float((st["w"][:nev] * np.einsum("ij,ij->j", X, BSX)).sum())


def test_gradient_full_size_vs_oracle_and_fd(g):
    """The 48^3 workload (n = 110,592, 49^3 cells), eigenvalue and eigenvector terms:
    every cell against the FP64 oracle's adjoint gradient (oracle eigenpairs), and the
    64 seeded cells against central differences of fresh solves, both to 1e-5 relative
    per cell (absolute floors only for cells whose gradient is near zero)."""
    N, nev, bs = 48, 10, 2
    st = W.q1grad_setup(N, seed=0, nev=nev)
    c0 = st["c"].copy()
    grad, ev, X, p = _gpu_grad(g, N, st, nev, bs, tol=1e-12, use_vec=True)
    # oracle: FP64 GCG eigenpairs and the adjoint formulas
    r = G.gcg(p.A, p.B, nev, bs, 1e-11, W.initial_block(p.n, nev + 3 * bs, 0))
    assert r.converged
    Sm = sp.diags(st["S"])
    BS = (Sm @ p.B @ Sm).tocsr()
    Gx = np.stack([2 * st["w"][i] * (BS @ r.evecs[:, i]) for i in range(nev)], axis=1)
    ref = GR.loss_grad_cells(N, p.A, p.B, r.evals, r.evecs, np.ones(nev), Gx, tol=1e-13)
    assert np.abs(ev - r.evals).max() <= 1e-10 * r.evals.max()
    scale = np.abs(ref).max()
    assert np.all(np.abs(grad - ref) <= 1e-5 * np.abs(ref) + 1e-9 * scale)
    # central differences on the 64 seeded cells, delta = 1e-3 c_e, solves at 1e-12
    cf = c0.ravel()
    for e in st["fd_cells"]:
        d = 1e-3 * cf[e]
        vals = []
        for sgn in (1, -1):
            cc = cf.copy()
            cc[e] += sgn * d
            vals.append(_loss_fd(g, N, st, cc.reshape(c0.shape), nev, bs, 1e-12))
        fd = (vals[0] - vals[1]) / (2 * d)
        assert abs(fd - grad[e]) <= 1e-5 * abs(grad[e]) + 2e-7, (e, fd, grad[e])
