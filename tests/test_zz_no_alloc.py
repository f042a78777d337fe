"""gcge_gram_f64_noalloc: the Gram product for callers that cannot allocate device memory.

Such callers (an application whose allocator has reserved the GPU's memory, or a
loop that cannot pay for cudaMalloc/cudaFree) use this entry point; it must give the
same result as gcge_gram_f64, call after call, even though every call reuses one
static scratch array inside the library.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _gram_pair(g, torch, n, m, k, seed, beta):
    rng = np.random.default_rng(seed)
    X = torch.tensor(rng.standard_normal((n, m)), device="cuda")
    Y = torch.tensor(rng.standard_normal((n, k)), device="cuda")
    C0 = rng.standard_normal((k, m + 3))            # column-major (m+3) x k, ldc = m + 3
    C_ref = torch.tensor(C0, device="cuda")
    C_new = torch.tensor(C0, device="cuda")
    g.gcge_gram_f64(n, m, k, 0.75, X, m, Y, k, beta, C_ref, m + 3)
    g.gcge_gram_f64_noalloc(n, m, k, 0.75, X, m, Y, k, beta, C_new, m + 3)
    torch.cuda.synchronize()
    return C_ref.cpu().numpy(), C_new.cpu().numpy()


def test_noalloc_gram_matches_allocating_entry_point_twice():
    import torch
    import paper_2111_06552_gb300 as g
    assert torch.cuda.is_available()
    # two calls in a row with different shapes: the second must not see the first's partials
    for (n, m, k, seed, beta) in ((70001, 150, 33, 1, 0.0), (5003, 20, 7, 2, 0.5)):
        ref, new = _gram_pair(g, torch, n, m, k, seed, beta)
        tol = 1e-12 * (np.abs(ref).max() + 1.0)
        assert np.abs(new - ref).max() <= tol
        # entries outside the m x k sub-block are untouched by both
        assert np.array_equal(new[:, m:], ref[:, m:])


def test_noalloc_gram_rejects_oversize():
    import torch
    import paper_2111_06552_gb300 as g
    big = g.GCGE_GRAM_NOALLOC_MAX_DOUBLES // 100 + 1
    Cm = torch.zeros(8, device="cuda", dtype=torch.float64)
    X = torch.zeros(8, device="cuda", dtype=torch.float64)
    s = g.lib().gcge_gram_f64_noalloc(1, big, 100, 1.0, X.data_ptr(), big, X.data_ptr(), 100, 0.0,
                                      Cm.data_ptr(), big, None)
    assert s == g.GCGE_EINVAL
    assert b"GCGE_GRAM_NOALLOC_MAX_DOUBLES" in g.lib().gcge_last_error_message()
