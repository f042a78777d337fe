"""Parity of each hot-path kernel (through the C ABI) with the FP64 oracle's step.

Sizes span several tiles and ragged tails; FP64 kernels must agree to rounding
(1e-12 relative), FP32 kernels to the FP32 bound stated per test.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import linalg as L
from oracle import cg as CG
from oracle import orth as O

from gpu_util import dev, csr_dev, padded, host, subspace_cos

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    import paper_2111_06552_gb300 as gg
    assert torch.cuda.is_available()
    gg.lib()
    return gg


def _ragged_csr(n, seed):
    """Symmetric random pattern with very uneven rows (1 .. ~60 entries) and an empty row."""
    rng = np.random.default_rng(seed)
    A = W.random_sparse_spd(n, 0.02, seed)
    rows = rng.choice(n, size=max(1, n // 50), replace=False)
    D = sp.random(n, n, density=0.0, format="lil")
    for r in rows:
        cols = rng.choice(n, size=min(n, 60), replace=False)
        D[r, cols] = rng.uniform(-1, 1, cols.size)
    A = (A + D.tocsr() + D.tocsr().T).tocsr()
    A.sort_indices()
    A = A.tolil()
    A[n // 3, :] = 0.0            # an empty row (structurally)
    A = A.tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    return A


@pytest.mark.parametrize("k", [1, 3, 10, 17, 20, 40, 100, 130])
def test_spmm_f64_matches_oracle(g, k):
    import torch
    n = 1237
    A = _ragged_csr(n, k)
    rng = np.random.default_rng(k)
    X = rng.standard_normal((n, k))
    Y0 = rng.standard_normal((n, k))
    ldx, ldy = k + 3, k + 1
    rp, ci, val = csr_dev(A)
    Xd = dev(padded(X, ldx))
    Yd = dev(padded(Y0, ldy))
    g.gcge_spmm_f64(n, rp, ci, val, k, 2.0, Xd, ldx, -0.5, Yd, ldy)
    torch.cuda.synchronize()
    ref = 2.0 * L.spmm(A, X) - 0.5 * Y0
    got = host(Yd)[:, :k]
    assert np.abs(got - ref).max() <= 1e-12 * (np.abs(ref).max() + 1)
    assert np.isnan(host(Yd)[:, k:]).all()           # padding untouched


@pytest.mark.parametrize("k", [2, 20, 40, 100])
def test_spmm_f32_matches_oracle(g, k):
    import torch
    p = W.make_config("q1_160", N=12, seed=1)
    A = p.A
    n = p.n
    X = np.random.default_rng(3).standard_normal((n, k)).astype(np.float32)
    rp, ci, val = csr_dev(A, f32=True)
    Xd = dev(X)
    Yd = torch.zeros((n, k), dtype=torch.float32, device="cuda")
    g.gcge_spmm_f32(n, rp, ci, val, k, 1.0, Xd, k, 0.0, Yd, k)
    torch.cuda.synchronize()
    ref = L.spmm(A.astype(np.float32).astype(np.float64), X.astype(np.float64))
    scale = abs(A).astype(np.float64) @ np.abs(X.astype(np.float64))
    assert np.all(np.abs(host(Yd) - ref) <= 2e-6 * scale + 1e-30)


@pytest.mark.parametrize("n,m,k", [(1, 1, 1), (1000, 7, 5), (4133, 70, 20), (20011, 150, 33),
                                   (3001, 200, 100), (20000, 10, 10), (5003, 20, 20),
                                   (3000, 13, 9)])
def test_gram_f64_into_strided_subblock(g, n, m, k):
    import torch
    rng = np.random.default_rng(n + m)
    X = rng.standard_normal((n, m))
    Y = rng.standard_normal((n, k))
    ldc, r0, c0 = m + 9, 4, 3
    Cbig = np.full((ldc, k + 6), 7.0)     # column-major ldc x (k+6) as a (k+6, ldc) C-order array
    Cd = dev(Cbig.T.copy())
    base = Cd.data_ptr() + 8 * (r0 + c0 * ldc)
    g.gcge_gram_f64(n, m, k, 1.5, dev(X), m, dev(Y), k, 0.5, base, ldc)
    torch.cuda.synchronize()
    got = host(Cd).T        # ldc x (k+6) column-major view
    ref = 1.5 * (X.T @ Y) + 0.5 * 7.0
    assert np.abs(got[r0:r0 + m, c0:c0 + k] - ref).max() <= 1e-12 * (np.abs(ref).max() + 1)
    mask = np.ones_like(got, dtype=bool)
    mask[r0:r0 + m, c0:c0 + k] = False
    assert np.all(got[mask] == 7.0)


@pytest.mark.parametrize("tc", [0, 1])
@pytest.mark.parametrize("n,m,k", [(5000, 70, 20), (20011, 150, 33), (65536 + 17, 96, 40)])
def test_gram_f32(g, n, m, k, tc):
    import torch
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, m)).astype(np.float32)
    Y = rng.standard_normal((n, k)).astype(np.float32)
    Cd = torch.zeros((k, m), dtype=torch.float64, device="cuda")   # col-major m x k
    g.gcge_gram_f32(n, m, k, 1.0, dev(X), m, dev(Y), k, 0.0, Cd, m, tc=tc)
    torch.cuda.synchronize()
    ref = X.astype(np.float64).T @ Y.astype(np.float64)
    bound = np.abs(X.astype(np.float64)).T @ np.abs(Y.astype(np.float64))
    assert np.all(np.abs(host(Cd).T - ref) <= 2e-6 * bound)


@pytest.mark.parametrize("n,d,q", [(1, 1, 1), (999, 13, 7), (10007, 200, 180), (4096, 70, 50),
                                   (20000, 10, 10), (385, 20, 20), (5000, 33, 65),
                                   (777, 17, 31), (1000, 0, 3)])
def test_vc_f64(g, n, d, q):
    import torch
    rng = np.random.default_rng(d)
    V = rng.standard_normal((n, d))
    Cm = rng.standard_normal((d, q))
    Y0 = rng.standard_normal((n, q))
    ldv, ldy, ldc = d + 2, q + 5, d + 1
    Cbuf = np.zeros((q, ldc))
    Cbuf[:, :d] = Cm.T                   # column-major d x q with ldc
    Yd = dev(padded(Y0, ldy))
    g.gcge_vc_f64(n, d, q, -1.0, dev(padded(V, ldv)), ldv, dev(Cbuf), ldc, 2.0, Yd, ldy)
    torch.cuda.synchronize()
    ref = -(V @ Cm) + 2.0 * Y0
    got = host(Yd)
    assert np.abs(got[:, :q] - ref).max() <= 1e-12 * (np.abs(ref).max() + 1)
    assert np.all(np.isnan(got[:, q:]))             # padding columns untouched


@pytest.mark.parametrize("tc", [0, 1])
def test_vc_f32(g, tc):
    import torch
    n, d, q = 33001, 120, 100
    rng = np.random.default_rng(0)
    V = rng.standard_normal((n, d)).astype(np.float32)
    Cm = rng.standard_normal((d, q))
    Yd = torch.zeros((n, q), dtype=torch.float32, device="cuda")
    g.gcge_vc_f32(n, d, q, 1.0, dev(V), d, dev(Cm.T.copy()), d, 0.0, Yd, q, tc=tc)
    torch.cuda.synchronize()
    ref = V.astype(np.float64) @ Cm
    bound = np.abs(V.astype(np.float64)) @ np.abs(Cm)
    assert np.all(np.abs(host(Yd) - ref) <= 2e-6 * bound + 1e-6)


@pytest.mark.parametrize("d", [1, 2, 3, 16, 17, 64, 70, 129, 200])
def test_syev_matches_oracle(g, d):
    import torch
    rng = np.random.default_rng(d)
    M = rng.standard_normal((d, d))
    M = M + M.T
    if d >= 16:   # include an exactly repeated eigenvalue and a wide spread
        Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
        lam = np.sort(rng.uniform(1, 1e4, d))
        lam[3:6] = lam[3]
        M = (Q * lam) @ Q.T
        M = 0.5 * (M + M.T)
    w_ref, _ = L.sym_eig(M)
    Ad = dev(M.T.copy())
    wd = torch.zeros(d, dtype=torch.float64, device="cuda")
    Qd = torch.zeros((d, d), dtype=torch.float64, device="cuda")
    sweeps = g.gcge_syev(d, Ad, d, wd, Qd, d)
    w = host(wd)
    Qh = host(Qd).T
    nrm = np.abs(w_ref).max()
    assert np.abs(w - w_ref).max() <= 1e-13 * nrm * max(1.0, np.sqrt(d) / 4)
    assert np.abs(Qh.T @ Qh - np.eye(d)).max() <= 1e-13 * d
    assert np.abs(M @ Qh - Qh * w).max() <= 1e-12 * nrm
    assert sweeps < 30


def _structured_abar(rng, nx, npp, nw, scale):
    """A Rayleigh-Ritz matrix with the structure of Eq. (struct_bar_A_new): diagonal Ritz
    values on the X block, zero X-P coupling, a dense P block and W coupled to both."""
    lam = np.sort(3 * np.pi ** 2 * (1 + 30 * rng.random(nx)))
    d = nx + npp + nw
    A = np.zeros((d, d))
    A[:nx, :nx] = np.diag(lam)
    M = rng.standard_normal((npp, npp))
    A[nx:nx + npp, nx:nx + npp] = lam[-1] * (M @ M.T / npp + np.eye(npp))
    Bx = scale * lam[:, None] * rng.standard_normal((nx, nw))
    A[:nx, nx + npp:] = Bx
    A[nx + npp:, :nx] = Bx.T
    Bp = scale * lam[-1] * rng.standard_normal((npp, nw))
    A[nx:nx + npp, nx + npp:] = Bp
    A[nx + npp:, nx:nx + npp] = Bp.T
    G = rng.standard_normal((nw, nw))
    A[nx + npp:, nx + npp:] = 2 * lam[-1] * (G @ G.T / nw + np.eye(nw))
    return A


@pytest.mark.parametrize("scale", [1e-1, 1e-4])
def test_syev_structured_rr_matrix_d500(g, scale):
    """The order of the first Rayleigh-Ritz matrix of the 160^3 workload (sizeX 300 +
    P 100 + W 100), with strong and weak coupling, against LAPACK."""
    import torch
    rng = np.random.default_rng(int(-np.log10(scale)))
    M = _structured_abar(rng, 300, 100, 100, scale)
    d = M.shape[0]
    w_ref, _ = L.sym_eig(M)
    wd = torch.zeros(d, dtype=torch.float64, device="cuda")
    Qd = torch.zeros((d, d), dtype=torch.float64, device="cuda")
    g.gcge_syev(d, dev(M.T.copy()), d, wd, Qd, d)
    w = host(wd)
    Qh = host(Qd).T
    nrm = np.abs(w_ref).max()
    assert np.abs(w - w_ref).max() <= 1e-13 * nrm * max(1.0, np.sqrt(d) / 4)
    assert np.abs(Qh.T @ Qh - np.eye(d)).max() <= 1e-13 * d
    assert np.abs(M @ Qh - Qh * w).max() <= 1e-12 * nrm


def test_syev_degenerate_and_diagonal(g):
    import torch
    for M in (np.eye(8), np.diag(np.arange(10.0)[::-1]), np.zeros((5, 5))):
        d = M.shape[0]
        wd = torch.zeros(d, dtype=torch.float64, device="cuda")
        Qd = torch.zeros((d, d), dtype=torch.float64, device="cuda")
        g.gcge_syev(d, dev(M.T.copy()), d, wd, Qd, d)
        assert np.allclose(host(wd), np.sort(np.diag(M)))


@pytest.mark.parametrize("theta", [0.0, 0.7])
def test_block_cg_matches_oracle(g, theta):
    import torch
    p = W.make_config("q1grad_48", N=9, seed=4)
    n = p.n
    rng = np.random.default_rng(1)
    k = 7
    X0 = rng.standard_normal((n, k))
    lam = np.linspace(20, 40, k)
    rhs = L.spmm(p.B, X0) * (lam - theta)
    S = CG.shifted_matrix(p.A, p.B, theta)
    for max_iter, rtol in ((4, 0.0), (30, 1e-2)):
        ref, it_ref, _ = CG.shifted_cg(p.A, p.B, theta, X0, lam, max_iter, rtol, rhs=rhs)
        rp, ci, val = csr_dev(S)
        Xd = dev(padded(X0, k + 1))
        it = g.gcge_block_cg_f64(n, rp, ci, val, k, dev(rhs), k, Xd, k + 1, max_iter, rtol)
        torch.cuda.synchronize()
        assert np.array_equal(it, it_ref)
        got = host(Xd)[:, :k]
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("theta", [0.0, 0.7])
def test_block_pcg_matches_oracle(g, theta):
    """Jacobi-preconditioned CG (M = |diag(S)|) on the lognormal FD pencil: identical
    per-column step counts and iterates to 1e-10 of the oracle's preconditioned CG."""
    import torch
    p = W.make_config("fd3d_128", N=10, seed=4)
    n = p.n
    k = 6
    X0 = np.random.default_rng(5).standard_normal((n, k))
    lam = np.linspace(20, 40, k)
    rhs = L.spmm(p.B, X0) * (lam - theta)
    S = CG.shifted_matrix(p.A, p.B, theta)
    for max_iter, rtol in ((5, 0.0), (40, 1e-2)):
        ref, it_ref, _ = CG.shifted_cg(p.A, p.B, theta, X0, lam, max_iter, rtol, rhs=rhs,
                                       precond=True)
        rp, ci, val = csr_dev(S)
        Xd = dev(padded(X0, k + 2))
        it = g.gcge_block_cg_f64(n, rp, ci, val, k, dev(rhs), k, Xd, k + 2, max_iter, rtol,
                                 precond=g.GCGE_PRECOND_JACOBI)
        torch.cuda.synchronize()
        assert np.array_equal(it, it_ref)
        got = host(Xd)[:, :k]
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_block_cg_f32(g):
    import torch
    p = W.make_config("fd3d_128", N=12, seed=2)
    n = p.n
    k = 5
    X0 = np.random.default_rng(2).standard_normal((n, k))
    lam = np.full(k, 10.0)
    rhs = L.spmm(p.B, X0) * lam
    ref, it_ref, _ = CG.shifted_cg(p.A, p.B, 0.0, X0, lam, 6, 0.0, rhs=rhs)
    rp, ci, val = csr_dev(p.A, f32=True)
    Xd = dev(X0.astype(np.float32))
    it = g.gcge_block_cg_f32(n, rp, ci, val, k, dev(rhs.astype(np.float32)), k, Xd, k, 6, 0.0)
    torch.cuda.synchronize()
    assert np.all(it == 6)
    assert np.abs(host(Xd) - ref).max() <= 2e-4 * np.abs(ref).max()


@pytest.mark.parametrize("orth", [0, 1])
@pytest.mark.parametrize("m,q", [(1, 0), (5, 0), (20, 6), (37, 11)])
def test_borth_matches_oracle(g, m, q, orth):
    import torch
    p = W.make_config("q1grad_48", N=8, seed=5)
    n = p.n
    rng = np.random.default_rng(m)
    Q0, _ = O.b_orthonormalize(rng.standard_normal((n, q)), None, p.B) if q else (None, None)
    X = rng.standard_normal((n, m))
    if m >= 5:
        X[:, 3] = X[:, 0] - 2 * X[:, 1]                   # dependent inside the block
    if q and m >= 5:
        X[:, 4] = Q0 @ rng.standard_normal(q)             # inside span(Q0)
    # orth 0: Algorithm 3 (RecursiveOrthSVD); 1: Algorithm 2 (modified block orthogonalisation)
    Y_ref, _ = (O.b_orthonormalize if orth == 0 else O.b_orthonormalize_alg2)(X, Q0, p.B)
    rp, ci, val = csr_dev(p.B)
    Wd = dev(padded(X, m))
    Qd = dev(Q0) if q else None
    mo = g.gcge_borth_f64(n, rp, ci, val, Qd, q if q else 1, q, Wd, m, m, 16, orth)
    torch.cuda.synchronize()
    assert mo == Y_ref.shape[1]
    Y = host(Wd)[:, :mo]
    BY = p.B @ Y
    assert np.abs(Y.T @ BY - np.eye(mo)).max() < 1e-12
    if q:
        assert np.abs(Q0.T @ BY).max() < 1e-12
    cos = subspace_cos(Y, Y_ref, p.B)
    assert cos.min() > 1 - 1e-10
    if orth == 1:   # Gram-Schmidt fixes the basis itself, column by column
        assert np.abs(Y - Y_ref).max() <= 1e-8 * np.abs(Y_ref).max()


def test_random_block_matches_generator(g):
    import torch
    n, k = 1001, 13
    Xd = torch.zeros((n, k + 3), dtype=torch.float64, device="cuda")
    g.gcge_random_block_f64(n, k, 12345, Xd, k + 3)
    torch.cuda.synchronize()
    ref = W.initial_block(n, k, 12345)
    assert np.abs(host(Xd)[:, :k] - ref).max() < 1e-12


@pytest.mark.parametrize("n,m,k,offx,offy,ldx,ldy", [
    (70001, 300, 150, 1, 3, 308, 156),   # 2 column groups of X, 2 of Y, unaligned bases
    (4099, 40, 7, 2, 0, 44, 8),          # one tile, narrow Y
    (129, 513, 1, 0, 1, 516, 4),         # few rows, 3 column groups, k = 1
    (20011, 150, 33, 1, 1, 151, 35),     # leading dimensions not multiples of 4
])
def test_gram_f32_tc_layouts(g, n, m, k, offx, offy, ldx, ldy):
    """Tensor-core Gram on sub-blocks of wider buffers (NaN outside the block)."""
    import torch
    rng = np.random.default_rng(n + m)
    X = rng.standard_normal((n, m)).astype(np.float32)
    Y = rng.standard_normal((n, k)).astype(np.float32)
    Xb = np.full((n, ldx), np.nan, np.float32)
    Xb[:, offx:offx + m] = X
    Yb = np.full((n, ldy), np.nan, np.float32)
    Yb[:, offy:offy + k] = Y
    Xd, Yd = dev(Xb), dev(Yb)
    ldc = m + 2
    Cd = torch.full((k, ldc), 5.0, dtype=torch.float64, device="cuda")   # col-major ldc x k
    g.gcge_gram_f32(n, m, k, 1.5, Xd.data_ptr() + 4 * offx, ldx, Yd.data_ptr() + 4 * offy, ldy,
                    0.5, Cd, ldc, tc=1)
    torch.cuda.synchronize()
    got = host(Cd).T
    ref = 1.5 * (X.astype(np.float64).T @ Y.astype(np.float64)) + 2.5
    bound = 1.5 * np.abs(X.astype(np.float64)).T @ np.abs(Y.astype(np.float64))
    assert np.all(np.abs(got[:m] - ref) <= 2e-6 * bound + 1e-12)
    assert np.all(got[m:] == 5.0)
    assert g.gcge_tc_status() == 0   # no bounded wait ran out


@pytest.mark.parametrize("n,d,q,offv,offy,ldv,ldy,beta", [
    (70001, 37, 300, 3, 1, 44, 308, 0.5),     # 2 column groups of the result, unaligned
    (1000, 200, 160, 0, 0, 200, 160, 0.0),
    (257, 5, 20, 1, 2, 8, 24, -1.0),          # d below one K chunk
    (33001, 120, 100, 1, 0, 121, 100, 0.0),   # ldv not a multiple of 4
])
def test_vc_f32_tc_layouts(g, n, d, q, offv, offy, ldv, ldy, beta):
    """Tensor-core V C on sub-blocks of wider buffers (NaN outside the blocks)."""
    import torch
    rng = np.random.default_rng(n + d)
    V = rng.standard_normal((n, d)).astype(np.float32)
    Cm = rng.standard_normal((d, q))
    Y0 = rng.standard_normal((n, q)).astype(np.float32)
    Vb = np.full((n, ldv), np.nan, np.float32)
    Vb[:, offv:offv + d] = V
    Yb = np.full((n, ldy), np.nan, np.float32)
    Yb[:, offy:offy + q] = Y0
    Vd, Yd = dev(Vb), dev(Yb)
    ldc = d + 3
    Cbuf = np.full((q, ldc), np.nan)
    Cbuf[:, :d] = Cm.T
    g.gcge_vc_f32(n, d, q, 2.0, Vd.data_ptr() + 4 * offv, ldv, dev(Cbuf), ldc, beta,
                  Yd.data_ptr() + 4 * offy, ldy, tc=1)
    torch.cuda.synchronize()
    got = host(Yd)
    ref = 2.0 * (V.astype(np.float64) @ Cm) + beta * Y0.astype(np.float64)
    bound = 2.0 * np.abs(V.astype(np.float64)) @ np.abs(Cm) + abs(beta) * np.abs(Y0)
    assert np.all(np.abs(got[:, offy:offy + q] - ref) <= 2e-6 * bound + 1e-6)
    mask = np.ones(got.shape, dtype=bool)
    mask[:, offy:offy + q] = False
    assert np.all(np.isnan(got[mask]))
    assert g.gcge_tc_status() == 0


def test_gram_f32_tc_long_rows(g):
    """Tensor-core Gram over 2^21 rows of non-zero-mean data: the FP32 accumulator is
    drained into FP64 in windows, so the error stays at FP32-product level instead of
    growing with the rows one CTA covers."""
    import torch
    n, m, k = 2097152, 40, 40
    gen = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(n, m, device="cuda", generator=gen) + 0.5
    Y = torch.randn(n, k, device="cuda", generator=gen) + 0.5
    C = torch.zeros(k, m, dtype=torch.float64, device="cuda")
    g.gcge_gram_f32(n, m, k, 1.0, X, m, Y, k, 0.0, C, m, tc=1)
    torch.cuda.synchronize()
    ref = X.double().T @ Y.double()
    bound = X.double().abs().T @ Y.double().abs()
    assert ((C.T - ref).abs() / bound).max().item() <= 2e-6
