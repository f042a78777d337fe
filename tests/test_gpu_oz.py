"""FP64 Gram and V C products on the bf16 tensor cores (gcge_gram_f64_tc, gcge_vc_f64_tc).

The kernels cut every operand, per window of 128 reduction entries and per row, into
seven signed 7-bit digits below one exponent, multiply digit planes exactly on the
tensor cores and sum each window in FP64.  Checks:
* integer data that the digits hold exactly: the result equals the exact sum bit for bit;
* full-precision data over a wide range of magnitudes: the error stays inside the
  error model 2^-45 * 128 * sum over windows of max|x| max|y| (exact reference from
  error-free products and math.fsum);
* random normal data: agreement with the FP64 kernel inside the same error model;
* shapes with ragged tails, several row and column tiles, strided sub-blocks,
  alpha/beta, zero columns.
"""
import math

import numpy as np
import pytest

from gpu_util import dev, padded, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    import paper_2111_06552_gb300 as gg
    assert torch.cuda.is_available()
    gg.lib()
    return gg


def _split(x):
    """Dekker split: x = hi + lo with 26-bit halves whose products are exact in FP64."""
    c = 134217729.0 * x
    hi = c - (c - x)
    return hi, x - hi


def _exact_dot(x, y):
    """Correctly rounded sum_r x_r y_r (error-free products, math.fsum)."""
    xh, xl = _split(x)
    yh, yl = _split(y)
    terms = np.concatenate([xh * yh, xh * yl, xl * yh, xl * yl])
    return math.fsum(terms.tolist())


def _window_bound(x, y, win=128):
    n = x.size
    b = 0.0
    for w0 in range(0, n, win):
        b += win * np.abs(x[w0:w0 + win]).max() * np.abs(y[w0:w0 + win]).max()
    return 2.0 ** -45 * b


def _window_max(A, win=128):
    """max |A| over windows of `win` rows, per column: shape (windows, columns)."""
    n = A.shape[0]
    return np.stack([np.abs(A[w0:w0 + win]).max(axis=0) for w0 in range(0, n, win)])


def _model_gram(X, Y, win=128):
    """sum over windows of win * max|x_a| max|y_b| (the unit of the error model)."""
    return win * (_window_max(X, win).T @ _window_max(Y, win))


def _gram_tc(g, X, Y, alpha=1.0, beta=0.0, C0=None, ldx=None, ldy=None):
    import torch
    n, m = X.shape
    k = Y.shape[1]
    ldx = ldx or m
    ldy = ldy or k
    Cd = torch.zeros((k, m), dtype=torch.float64, device="cuda") if C0 is None else dev(C0.T.copy())
    g.gcge_gram_f64_tc(n, m, k, alpha, dev(padded(X, ldx)), ldx, dev(padded(Y, ldy)), ldy, beta,
                       Cd, m)
    torch.cuda.synchronize()
    g.gcge_tc_status()
    return host(Cd).T


@pytest.mark.parametrize("n,m,k", [(1, 1, 1), (300, 5, 3), (70001, 130, 37), (4096, 64, 100)])
def test_gram_tc_exact_on_integers(g, n, m, k):
    rng = np.random.default_rng(n + m + k)
    X = rng.integers(-2 ** 15, 2 ** 15, size=(n, m)).astype(np.float64)
    Y = rng.integers(-2 ** 15, 2 ** 15, size=(n, k)).astype(np.float64)
    X[:, 0] = 0.0                                   # a zero column
    got = _gram_tc(g, X, Y)
    assert np.array_equal(got, X.T @ Y)            # every partial sum is an exact integer


@pytest.mark.parametrize("n,m,k", [(3000, 9, 5), (1029, 140, 66)])
def test_gram_tc_error_model_wide_range(g, n, m, k):
    rng = np.random.default_rng(7 * n + k)
    X = rng.standard_normal((n, m)) * np.exp2(rng.integers(-30, 30, size=(n, 1)))
    Y = rng.standard_normal((n, k)) * np.exp2(rng.integers(-30, 30, size=(n, 1)))
    got = _gram_tc(g, X, Y, ldx=m + 3, ldy=k + 1)
    for a in range(0, m, max(1, m // 9)):
        for b in range(0, k, max(1, k // 5)):
            ref = _exact_dot(X[:, a], Y[:, b])
            assert abs(got[a, b] - ref) <= _window_bound(X[:, a], Y[:, b]), (a, b)


@pytest.mark.parametrize("n,m,k", [(262144 + 33, 200, 20), (50000, 400, 100)])
def test_gram_tc_matches_fp64_kernel(g, n, m, k):
    import torch
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, m))
    Y = rng.standard_normal((n, k))
    C0 = rng.standard_normal((m, k))
    got = _gram_tc(g, X, Y, alpha=-1.5, beta=0.25, C0=C0)
    Cd = dev(C0.T.copy())
    g.gcge_gram_f64(n, m, k, -1.5, dev(X), m, dev(Y), k, 0.25, Cd, m)
    torch.cuda.synchronize()
    ref = host(Cd).T
    # error model of the emulated product (window maxima) plus the FP64 kernel's own
    # rounding (1e-15 of sum |x||y| covers sqrt(n) eps at these sizes)
    model = 1.5 * 2.0 ** -45 * _model_gram(X, Y)
    bound = model + 1.5e-15 * (np.abs(X).T @ np.abs(Y)) + 1e-15 * np.abs(C0)
    assert np.all(np.abs(got - ref) <= bound)
    # and on random data the result is far inside FP64-level agreement
    assert np.abs(got - ref).max() <= 1e-14 * (np.abs(X).T @ np.abs(Y)).max()


def _vc_tc(g, V, Cm, alpha, beta, Y0, ldv, ldc, ldy):
    import torch
    n, d = V.shape
    q = Cm.shape[1]
    Cbuf = np.zeros((q, ldc))
    Cbuf[:, :d] = Cm.T
    Yd = dev(padded(Y0, ldy))
    g.gcge_vc_f64_tc(n, d, q, alpha, dev(padded(V, ldv)), ldv, dev(Cbuf), ldc, beta, Yd, ldy)
    torch.cuda.synchronize()
    g.gcge_tc_status()
    return host(Yd)


@pytest.mark.parametrize("n,d,q", [(1, 1, 1), (999, 13, 7), (10007, 300, 100), (4096, 64, 65)])
def test_vc_tc_exact_on_integers(g, n, d, q):
    rng = np.random.default_rng(d + q)
    V = rng.integers(-2 ** 15, 2 ** 15, size=(n, d)).astype(np.float64)
    Cm = rng.integers(-2 ** 15, 2 ** 15, size=(d, q)).astype(np.float64)
    Y0 = rng.integers(-2 ** 10, 2 ** 10, size=(n, q)).astype(np.float64)
    got = _vc_tc(g, V, Cm, 1.0, 2.0, Y0, d + 2, d + 1, q + 5)
    assert np.array_equal(got[:, :q], V @ Cm + 2.0 * Y0)
    assert np.all(np.isnan(got[:, q:]))             # padding columns untouched


@pytest.mark.parametrize("n,d,q", [(20000, 500, 300), (5000, 37, 129)])
def test_vc_tc_matches_fp64_kernel(g, n, d, q):
    import torch
    rng = np.random.default_rng(q)
    V = rng.standard_normal((n, d)) * np.exp2(rng.integers(-20, 20, size=(n, 1)))
    Cm = rng.standard_normal((d, q))
    Y0 = rng.standard_normal((n, q))
    got = _vc_tc(g, V, Cm, -0.5, 1.5, Y0, d, d, q)[:, :q]
    ref = -0.5 * (V @ Cm) + 1.5 * Y0
    # error model: 2^-45 * 128 * sum over windows of the window maxima of V's row and
    # C's column, plus FP64 rounding of the reference and of alpha/beta
    model = 0.5 * 2.0 ** -45 * _model_gram(V.T, Cm)
    bound = model + 1e-15 * (0.5 * (np.abs(V) @ np.abs(Cm)) + 1.5 * np.abs(Y0))
    assert np.all(np.abs(got - ref) <= bound)
