"""Seeded synthetic inputs for the GCG eigensolver: matrices and initial blocks.

This module builds *inputs* only.  It holds none of the eigensolver's arithmetic
and is the one module shared by the CUDA path's tests/benchmark and by the CPU
oracle.  Every generator is deterministic in its seed.

Workloads (each is a sparse symmetric pencil (A, B), A symmetric, B SPD, the
problem class of Section 2, Eq. (1) of the GCGE paper):

* ``fd2d(N)``            5-point finite differences of -Laplace on the unit square,
                         N x N interior nodes, h = 1/(N+1), B = I.
* ``q1_kron(N)``         trilinear (Q1) finite elements of -Laplace on the unit cube,
                         N^3 interior nodes, A = K(x)M(x)M + M(x)K(x)M + M(x)M(x)K,
                         B = M(x)M(x)M with the 1D stiffness K = h^-1 tridiag(-1,2,-1)
                         and mass M = (h/6) tridiag(1,4,1)  (27 nonzeros per row).
* ``q1_var(N, c)``       the same Q1 discretisation with a per-cell coefficient
                         c_e on the (N+1)^3 cells, assembled element by element;
                         B is the coefficient-free consistent mass.
* ``fd3d_var(N, c, d)``  7-point finite-volume diffusion on N^3 nodes with a per-node
                         coefficient, harmonic-mean face coefficients, Dirichlet
                         ghosts taking the node's own coefficient, and a diagonal
                         (lumped) mass B = diag(d).

Node ordering everywhere is lexicographic with the first axis slowest:
p = (i0 * N + i1) * N + i2 (2D: p = i0 * N + i1).  CSR column indices are
sorted within each row and stored as int32.

``initial_block`` draws the N(0,1) starting block from a counter-based
generator (splitmix64 -> two uniforms -> Box-Muller) so that a GPU
implementation can reproduce the same block from the seed without a host copy.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "Pencil", "fd2d", "q1_kron", "q1_var", "fd3d_var", "random_sparse_spd",
    "lognormal_cells", "initial_block", "splitmix64", "CONFIGS", "make_config",
    "fd2d_eigs", "q1_eigs", "fd3d_eigs_const", "q1_cell_nodes", "q1_cell_jacobian",
    "q1grad_setup",
]


@dataclass
class Pencil:
    """A sparse symmetric pencil in CSR form (B may be None for B = I)."""
    A: sp.csr_matrix
    B: sp.csr_matrix | None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]


def _csr(m) -> sp.csr_matrix:
    m = sp.csr_matrix(m)
    m.sum_duplicates()
    m.sort_indices()
    m.indices = m.indices.astype(np.int32)
    m.indptr = m.indptr.astype(np.int32) if m.nnz < 2**31 else m.indptr
    return m


def _tridiag(N: int, lo: float, di: float) -> sp.csr_matrix:
    e = np.ones(N)
    return sp.diags([lo * e[:-1], di * e, lo * e[:-1]], [-1, 0, 1], format="csr")


# ----------------------------------------------------------------------------
# 2D finite differences
# ----------------------------------------------------------------------------
def fd2d(N: int) -> Pencil:
    """5-point -Laplace on N x N interior nodes, Dirichlet, h = 1/(N+1); B = I."""
    h = 1.0 / (N + 1)
    T = _tridiag(N, -1.0, 2.0)
    I = sp.identity(N, format="csr")
    A = (sp.kron(T, I) + sp.kron(I, T)) / (h * h)
    return Pencil(_csr(A), None, f"fd2d_{N}", {"N": N, "h": h})


def fd2d_eigs(N: int, count: int | None = None) -> np.ndarray:
    """Closed-form spectrum (4/h^2)(sin^2(i pi h/2) + sin^2(j pi h/2)), ascending."""
    h = 1.0 / (N + 1)
    k = np.arange(1, N + 1)
    s = (4.0 / (h * h)) * np.sin(k * math.pi * h / 2.0) ** 2
    ev = np.sort((s[:, None] + s[None, :]).ravel())
    return ev if count is None else ev[:count]


# ----------------------------------------------------------------------------
# 3D trilinear (Q1) finite elements
# ----------------------------------------------------------------------------
def q1_kron(N: int) -> Pencil:
    """Q1 stiffness/mass on N^3 interior nodes of the unit cube as Kronecker sums.

    A = K(x)M(x)M + M(x)K(x)M + M(x)M(x)K, B = M(x)M(x)M with K = h^-1 tridiag(-1,2,-1),
    M = (h/6) tridiag(1,4,1).  Entries are evaluated per stencil offset from the 1D
    factors and stored on the full 27-point pattern (the face couplings of A are
    exactly zero but kept, so A and B share one pattern).
    """
    h = 1.0 / (N + 1)
    K1 = {-1: -1.0 / h, 0: 2.0 / h, 1: -1.0 / h}
    M1 = {-1: h / 6.0, 0: 4.0 * h / 6.0, 1: h / 6.0}
    offs = [(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)]
    valsA = np.zeros((27, N, N, N))
    valsB = np.zeros((27, N, N, N))
    for t, (d0, d1, d2) in enumerate(offs):
        valsA[t] = (K1[d0] * M1[d1] * M1[d2] + M1[d0] * K1[d1] * M1[d2]
                    + M1[d0] * M1[d1] * K1[d2])
        valsB[t] = M1[d0] * M1[d1] * M1[d2]
    A, B = _stencil_to_csr(N, offs, valsA, valsB)
    return Pencil(A, B, f"q1_{N}", {"N": N, "h": h})


def q1_1d_eigs(N: int) -> np.ndarray:
    """1D generalized eigenvalues of K v = mu M v: (6/h^2)(1-cos k pi h)/(2+cos k pi h)."""
    h = 1.0 / (N + 1)
    c = np.cos(np.arange(1, N + 1) * math.pi * h)
    return (6.0 / (h * h)) * (1.0 - c) / (2.0 + c)


def q1_eigs(N: int, count: int | None = None) -> np.ndarray:
    """Closed-form 3D spectrum mu_i + mu_j + mu_k of the Kronecker Q1 pencil."""
    mu = q1_1d_eigs(N)
    # only the lowest few per axis can enter the lowest `count` sums
    m = N if count is None else min(N, count)
    mu = mu[:m]
    ev = np.sort((mu[:, None, None] + mu[None, :, None] + mu[None, None, :]).ravel())
    return ev if count is None else ev[:count]


def _q1_local():
    """1D element stiffness (times h) and mass (divided by h) on a cell of size h."""
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]])       # times 1/h
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0    # times h
    return k1, m1


def q1_var(N: int, c: np.ndarray | None = None) -> Pencil:
    """Q1 pencil with per-cell coefficient c (shape (N+1)^3), assembled by elements.

    A = sum_e c_e P_e^T Khat P_e, with Khat the trilinear cell stiffness
    h (k(x)m(x)m + m(x)k(x)m + m(x)m(x)k) (k = h^-1 [[1,-1],[-1,1]], m = h/6 [[2,1],[1,2]]);
    B = sum_e P_e^T (m(x)m(x)m) P_e.  Dirichlet nodes are dropped by P_e.
    With c == 1 this reproduces ``q1_kron`` up to rounding.
    """
    h = 1.0 / (N + 1)
    if c is None:
        c = np.ones((N + 1,) * 3)
    c = np.asarray(c, dtype=np.float64).reshape((N + 1,) * 3)
    k1, m1 = _q1_local()
    n = N ** 3
    offs = [(a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1)]
    valsA = np.zeros((27, N, N, N))
    valsB = np.zeros((27, N, N, N))
    for t, dl in enumerate(offs):
        # local corner a in {0,1}^3 of node p inside cell e = i + 1 - a; q = p + dl has b = a + dl
        for a0 in (0, 1):
            b0 = a0 + dl[0]
            if b0 not in (0, 1):
                continue
            for a1 in (0, 1):
                b1 = a1 + dl[1]
                if b1 not in (0, 1):
                    continue
                for a2 in (0, 1):
                    b2 = a2 + dl[2]
                    if b2 not in (0, 1):
                        continue
                    kA = h * (k1[a0, b0] * m1[a1, b1] * m1[a2, b2]
                              + m1[a0, b0] * k1[a1, b1] * m1[a2, b2]
                              + m1[a0, b0] * m1[a1, b1] * k1[a2, b2])
                    kB = h ** 3 * m1[a0, b0] * m1[a1, b1] * m1[a2, b2]
                    ce = c[1 - a0:1 - a0 + N, 1 - a1:1 - a1 + N, 1 - a2:1 - a2 + N]
                    valsA[t] += kA * ce
                    valsB[t] += kB
    return Pencil(*_stencil_to_csr(N, offs, valsA, valsB), f"q1var_{N}", {"N": N, "h": h})


def _stencil_to_csr(N, offs, valsA, valsB):
    """Pack per-offset value planes (len(offs), N, N, N) into CSR with sorted columns."""
    n = N ** 3
    idx = np.arange(N)
    I0, I1, I2 = np.meshgrid(idx, idx, idx, indexing="ij")
    nb = len(offs)
    cols = np.empty((nb, N, N, N), dtype=np.int64)
    mask = np.empty((nb, N, N, N), dtype=bool)
    for t, (d0, d1, d2) in enumerate(offs):
        j0, j1, j2 = I0 + d0, I1 + d1, I2 + d2
        mask[t] = (j0 >= 0) & (j0 < N) & (j1 >= 0) & (j1 < N) & (j2 >= 0) & (j2 < N)
        cols[t] = (j0 * N + j1) * N + j2
    # offsets are listed in increasing lexicographic order -> sorted columns per row
    mask = mask.reshape(nb, n).T
    cols = cols.reshape(nb, n).T[mask]
    counts = mask.sum(axis=1)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    out = []
    for vals in (valsA, valsB):
        if vals is None:
            out.append(None)
            continue
        v = vals.reshape(nb, n).T[mask]
        m = sp.csr_matrix((v, cols.astype(np.int32), indptr.astype(np.int32)), shape=(n, n))
        m.has_sorted_indices = True
        out.append(m)
    return out


def q1_cell_nodes(N: int) -> np.ndarray:
    """(N+1)^3 x 8 interior-node indices of every Q1 cell (-1 for Dirichlet nodes).

    Local node a = a0*4 + a1*2 + a2 of cell e = (e0, e1, e2) is node (e0+a0-1, ...).
    """
    e = np.arange(N + 1)
    E0, E1, E2 = np.meshgrid(e, e, e, indexing="ij")
    out = np.empty(((N + 1) ** 3, 8), dtype=np.int64)
    for a0 in (0, 1):
        for a1 in (0, 1):
            for a2 in (0, 1):
                i0, i1, i2 = E0 + a0 - 1, E1 + a1 - 1, E2 + a2 - 1
                ok = (i0 >= 0) & (i0 < N) & (i1 >= 0) & (i1 < N) & (i2 >= 0) & (i2 < N)
                out[:, a0 * 4 + a1 * 2 + a2] = np.where(ok, (i0 * N + i1) * N + i2, -1).ravel()
    return out


def q1_cell_jacobian(N: int, A: sp.csr_matrix) -> sp.csr_matrix:
    """J (nnz x (N+1)^3) with A(c).data = J @ c for the Q1 pencil of ``q1_var``.

    Row t of J belongs to the t-th stored nonzero (p, q) of A's CSR pattern; entry
    (t, e) is the cell stiffness Khat_e[a, b] of the local pair that maps to (p, q).
    """
    h = 1.0 / (N + 1)
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
    Khat = h * (np.kron(k1, np.kron(m1, m1)) + np.kron(m1, np.kron(k1, m1))
                + np.kron(m1, np.kron(m1, k1)))
    nodes = q1_cell_nodes(N)
    n = A.shape[0]
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(A.indptr))
    keys = rows * n + A.indices.astype(np.int64)
    ri, ci, vi = [], [], []
    cells = np.arange(nodes.shape[0])
    for a in range(8):
        for b in range(8):
            p, q = nodes[:, a], nodes[:, b]
            ok = (p >= 0) & (q >= 0)
            pos = np.searchsorted(keys, p[ok] * n + q[ok])
            ri.append(pos)
            ci.append(cells[ok])
            vi.append(np.full(pos.size, Khat[a, b]))
    J = sp.csr_matrix((np.concatenate(vi), (np.concatenate(ri), np.concatenate(ci))),
                      shape=(A.nnz, nodes.shape[0]))
    J.sum_duplicates()
    J.sort_indices()
    return J


# ----------------------------------------------------------------------------
# 3D 7-point finite-volume diffusion with variable coefficient
# ----------------------------------------------------------------------------
def fd3d_var(N: int, c: np.ndarray | None = None, d: np.ndarray | None = None) -> Pencil:
    """7-point flux-form -div(c grad u) on N^3 nodes, h = 1/(N+1).

    Face coefficient between nodes p and q is the harmonic mean 2 c_p c_q/(c_p+c_q);
    a face to a Dirichlet ghost takes c_p.  A = h^-2 (flux form).  B = diag(d)
    (identity when d is None).
    """
    h = 1.0 / (N + 1)
    if c is None:
        c = np.ones((N, N, N))
    c = np.asarray(c, dtype=np.float64).reshape(N, N, N)
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    vals = np.zeros((7, N, N, N))
    diag = np.zeros((N, N, N))
    for t, dl in enumerate(offs):
        if dl == (0, 0, 0):
            continue
        # neighbour coefficient with ghost = own coefficient
        cn = c.copy()
        src = [slice(None)] * 3
        dst = [slice(None)] * 3
        ax = [i for i in range(3) if dl[i] != 0][0]
        s = dl[ax]
        if s > 0:
            dst[ax] = slice(0, N - 1)
            src[ax] = slice(1, N)
        else:
            dst[ax] = slice(1, N)
            src[ax] = slice(0, N - 1)
        cn[tuple(dst)] = c[tuple(src)]
        cf = 2.0 * c * cn / (c + cn)
        diag += cf
        vals[t] = -cf
    vals[3] = diag
    vals /= h * h
    A, _ = _stencil_to_csr(N, offs, vals, None)
    B = None
    if d is not None:
        B = _csr(sp.diags(np.asarray(d, dtype=np.float64).ravel()))
    return Pencil(A, B, f"fd3d_{N}", {"N": N, "h": h})


def fd3d_eigs_const(N: int, count: int | None = None) -> np.ndarray:
    """Closed form for fd3d_var with c == 1, B = I: (4/h^2) sum_d sin^2(k_d pi h / 2)."""
    h = 1.0 / (N + 1)
    m = N if count is None else min(N, count)
    s = (4.0 / (h * h)) * np.sin(np.arange(1, m + 1) * math.pi * h / 2.0) ** 2
    ev = np.sort((s[:, None, None] + s[None, :, None] + s[None, None, :]).ravel())
    return ev if count is None else ev[:count]


# ----------------------------------------------------------------------------
# random fields and small random pencils
# ----------------------------------------------------------------------------
def lognormal_cells(shape, sigma: float, seed: int) -> np.ndarray:
    """exp(sigma * N(0,1)) per cell from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal(shape))


def random_sparse_spd(n: int, density: float, seed: int, shift: float = 0.5,
                      spd: bool = True) -> sp.csr_matrix:
    """Random sparse symmetric matrix with a random pattern (diagonal always present).

    With spd=True a diagonal shift makes it diagonally dominant (hence SPD);
    otherwise it is symmetric indefinite.
    """
    rng = np.random.default_rng(seed)
    R = sp.random(n, n, density=density, random_state=rng, format="csr")
    R.data = rng.uniform(-1.0, 1.0, R.nnz)
    S = (R + R.T) * 0.5
    rowsum = np.asarray(abs(S).sum(axis=1)).ravel()
    if spd:
        D = sp.diags(rowsum + shift + rng.uniform(0.0, 1.0, n))
    else:
        D = sp.diags(rng.uniform(-2.0, 2.0, n))
    return _csr(S + D)


# ----------------------------------------------------------------------------
# counter-based initial block
# ----------------------------------------------------------------------------
_M64 = (1 << 64) - 1
_GOLD = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(z: np.ndarray) -> np.ndarray:
    """The splitmix64 finaliser applied elementwise to uint64 counters (z + golden)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(z, dtype=np.uint64) + _GOLD).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def initial_block(n: int, k: int, seed: int, rows: slice | None = None) -> np.ndarray:
    """N(0,1) block, row-major n x k, entry (i, j) from counter c = i*k + j.

    key = splitmix64(seed); u1 = (splitmix64(key + 2c) >> 11 + 0.5) 2^-53,
    u2 likewise from 2c+1; z = sqrt(-2 ln u1) cos(2 pi u2).
    ``rows`` selects a row range (for sampling large blocks).
    """
    r0, r1 = (0, n) if rows is None else (rows.start or 0, rows.stop)
    key = splitmix64(np.array([seed], dtype=np.uint64))[0]
    c = (np.arange(r0, r1, dtype=np.uint64)[:, None] * np.uint64(k)
         + np.arange(k, dtype=np.uint64)[None, :])
    with np.errstate(over="ignore"):
        a = splitmix64(key + np.uint64(2) * c)
        b = splitmix64(key + np.uint64(2) * c + np.uint64(1))
    u1 = ((a >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = ((b >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# the five synthetic configurations
# ----------------------------------------------------------------------------
CONFIGS = {
    # name: (builder description, nev, block_size)
    "fd2d_64": dict(nev=20, bs=10),
    "q1_64": dict(nev=100, bs=20),
    "fd3d_128": dict(nev=200, bs=40),
    "q1grad_48": dict(nev=10, bs=2),
    "q1_160": dict(nev=1000, bs=100),
    # stand-in for the paper's SuiteSparse (PARSEC) class: random symmetric pattern,
    # about 60 nonzeros per row, diagonally dominant, B = I
    "rand_200k": dict(nev=50, bs=10),
}


def q1grad_setup(N: int, seed: int, nev: int = 10, sub: int = 8, n_fd: int = 64) -> dict:
    """Loss ingredients of the differentiation workload (Q1 on N^3, lognormal c):
    c (cells), the 0/1 node indicator of a seeded sub^3 node block S, weights w ~ U(0,1)
    for the eigenvector terms, and n_fd seeded cells for finite-difference checks.
    L = sum_i lambda_i + sum_i w_i x_i^T B_S x_i with B_S = D_S B D_S."""
    rng = np.random.default_rng(seed + 1000)
    c = lognormal_cells((N + 1,) * 3, 0.5, seed)
    sub = min(sub, N)
    o = rng.integers(0, N - sub + 1, size=3)
    mask = np.zeros((N, N, N))
    mask[o[0]:o[0] + sub, o[1]:o[1] + sub, o[2]:o[2] + sub] = 1.0
    w = rng.uniform(0.0, 1.0, nev)
    fd = rng.choice((N + 1) ** 3, size=min(n_fd, (N + 1) ** 3), replace=False)
    return {"c": c, "S": mask.ravel(), "w": w, "fd_cells": fd}


def make_config(name: str, seed: int = 0, N: int | None = None) -> Pencil:
    """Build one of the synthetic workloads (optionally at a reduced grid size N)."""
    if name.startswith("fd2d"):
        p = fd2d(N or 64)
    elif name == "q1_64" or name.startswith("q1kron"):
        p = q1_kron(N or 64)
    elif name.startswith("fd3d"):
        NN = N or 128
        rng = np.random.default_rng(seed)
        c = np.exp(rng.standard_normal((NN, NN, NN)))
        d = 1.0 + 0.1 * rng.uniform(-1.0, 1.0, NN ** 3)
        p = fd3d_var(NN, c, d)
    elif name.startswith("q1grad"):
        NN = N or 48
        c = lognormal_cells((NN + 1,) * 3, 0.5, seed)
        p = q1_var(NN, c)
        p.meta["c"] = c
    elif name.startswith("rand"):
        NN = N or 200000
        A = random_sparse_spd(NN, 30.0 / NN, seed)   # ~30 + 30 mirrored + diagonal per row
        p = Pencil(A, None, name, {"N": NN})
    elif name.startswith("q1_160") or name.startswith("q1var"):
        NN = N or 160
        c = lognormal_cells((NN + 1,) * 3, 1.0, seed)
        p = q1_var(NN, c)
        p.meta["c"] = c
    else:
        raise KeyError(name)
    p.meta.update(CONFIGS.get(name, {}))
    p.meta["seed"] = seed
    p.name = name if N is None else f"{name}@{N}"
    return p
