"""Input generators: sizes, symmetry, assembly identities and closed-form spectra."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_config_sizes_match_stencil_counts():
    sizes = json.load(open(os.path.join(GOLD, "config_sizes.json")))
    # build the small/medium ones; the 160^3 count is checked by formula on a reduced grid
    for name in ("fd2d_64", "q1_64", "q1grad_48"):
        p = W.make_config(name)
        assert p.n == sizes[name]["n"] and p.A.nnz == sizes[name]["nnz"], name
        assert W.CONFIGS[name]["nev"] == sizes[name]["nev"]
        assert W.CONFIGS[name]["bs"] == sizes[name]["bs"]
    p = W.make_config("fd3d_128", N=20)
    assert p.A.nnz == 7 * 20 ** 3 - 6 * 20 ** 2
    p = W.make_config("q1_160", N=12)
    assert p.A.nnz == (3 * 12 - 2) ** 3 == p.B.nnz


@pytest.mark.parametrize("name,N", [("fd2d_64", 9), ("q1_64", 5), ("fd3d_128", 6),
                                    ("q1grad_48", 5), ("q1_160", 4)])
def test_symmetric_and_sorted(name, N):
    p = W.make_config(name, N=N)
    for M in (p.A, p.B):
        if M is None:
            continue
        assert abs(M - M.T).max() <= 1e-14 * abs(M).max()
        for r in range(M.shape[0]):
            cols = M.indices[M.indptr[r]:M.indptr[r + 1]]
            assert np.all(np.diff(cols) > 0)
        assert M.indices.dtype == np.int32


def test_q1_element_assembly_reproduces_kronecker():
    N = 7
    h = 1.0 / (N + 1)
    K = (sp.diags([-np.ones(N - 1), 2 * np.ones(N), -np.ones(N - 1)], [-1, 0, 1])) / h
    M = (sp.diags([np.ones(N - 1), 4 * np.ones(N), np.ones(N - 1)], [-1, 0, 1])) * h / 6
    Ak = (sp.kron(K, sp.kron(M, M)) + sp.kron(M, sp.kron(K, M)) + sp.kron(M, sp.kron(M, K))).toarray()
    Bk = sp.kron(M, sp.kron(M, M)).toarray()
    pv = W.q1_var(N)
    pk = W.q1_kron(N)
    assert np.abs(pv.A.toarray() - Ak).max() <= 1e-14 * np.abs(Ak).max()
    assert np.abs(pv.B.toarray() - Bk).max() <= 1e-14 * np.abs(Bk).max()
    assert np.abs(pk.A.toarray() - Ak).max() <= 1e-14 * np.abs(Ak).max()


def test_q1_var_linear_in_coefficient():
    N = 4
    c1 = W.lognormal_cells((N + 1,) * 3, 1.0, 1)
    c2 = W.lognormal_cells((N + 1,) * 3, 1.0, 2)
    A1, A2 = W.q1_var(N, c1).A, W.q1_var(N, c2).A
    A12 = W.q1_var(N, 2.0 * c1 + 3.0 * c2).A
    assert abs(A12 - (2 * A1 + 3 * A2)).max() <= 1e-13 * abs(A12).max()


def test_closed_form_spectra():
    p = W.fd2d(9)
    ev = np.linalg.eigvalsh(p.A.toarray())
    assert np.allclose(ev, W.fd2d_eigs(9), rtol=1e-12, atol=0)
    p = W.q1_kron(6)
    ev = sl.eigh(p.A.toarray(), p.B.toarray(), eigvals_only=True)
    assert np.allclose(ev[:40], W.q1_eigs(6, 40), rtol=1e-12, atol=0)
    p = W.fd3d_var(6)
    ev = np.linalg.eigvalsh(p.A.toarray())
    assert np.allclose(ev[:40], W.fd3d_eigs_const(6, 40), rtol=1e-12, atol=0)
    # continuum limits quoted for the two closed-form configurations
    assert abs(W.fd2d_eigs(64, 1)[0] - 19.7353665) < 1e-6
    assert abs(W.q1_eigs(64, 1)[0] - 29.61457750) < 1e-7


def test_cut_cluster_in_q1_64():
    ev = W.q1_eigs(64, 110)
    # eigenvalues 97..102 (1-based) form one 6-fold cluster (permutations of (1,4,5))
    assert np.ptp(ev[96:102]) <= 1e-10 * ev[96]
    assert ev[95] < ev[96] * (1 - 1e-6) and ev[102] > ev[101] * (1 + 1e-6)


def test_initial_block_deterministic_and_normal():
    a = W.initial_block(2000, 7, 5)
    b = W.initial_block(2000, 7, 5)
    c = W.initial_block(2000, 7, 6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert abs(a.mean()) < 0.05 and abs(a.std() - 1.0) < 0.05
    part = W.initial_block(2000, 7, 5, rows=slice(100, 130))
    assert np.array_equal(part, a[100:130])


def test_splitmix64_reference_values():
    # splitmix64 with state 0: the first outputs of the published generator
    z = np.array([0], dtype=np.uint64)
    assert int(W.splitmix64(z)[0]) == 0xE220A8397B1DCDAF
    z = np.array([0x9E3779B97F4A7C15], dtype=np.uint64)
    assert int(W.splitmix64(z)[0]) == 0x6E789E6AA1B965F4


def test_random_pattern_stand_in():
    """The SuiteSparse-class stand-in: symmetric, ~61 nonzeros per row, SPD by
    diagonal dominance, deterministic in its seed."""
    p = W.make_config("rand_200k", N=4000, seed=2)
    A = p.A
    assert p.B is None and A.shape == (4000, 4000)
    assert abs(A.nnz / A.shape[0] - 61) < 3
    assert abs(A - A.T).max() == 0.0
    off = abs(A).sum(axis=1).A.ravel() - abs(A.diagonal())
    assert np.all(A.diagonal() > off)              # strictly diagonally dominant
    q = W.make_config("rand_200k", N=4000, seed=2)
    assert np.array_equal(q.A.data, A.data) and np.array_equal(q.A.indices, A.indices)
