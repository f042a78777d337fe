"""Helpers for the GPU parity tests: device copies of seeded inputs."""
import numpy as np


def torch_mod():
    import torch
    return torch


def dev(a, dtype=None):
    torch = torch_mod()
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def csr_dev(M, f32=False):
    torch = torch_mod()
    rp = dev(M.indptr.astype(np.int32))
    ci = dev(M.indices.astype(np.int32))
    val = dev(M.data.astype(np.float32 if f32 else np.float64))
    return rp, ci, val


def padded(X, ld, dtype=np.float64):
    """Row-major n x k block stored with leading dimension ld (extra columns = NaN guard)."""
    n, k = X.shape
    out = np.full((n, ld), np.nan, dtype=dtype)
    out[:, :k] = X
    return out


def host(t):
    return t.detach().cpu().numpy()


def subspace_cos(X, Y, B=None):
    """Cosines of the principal angles between span(X) and span(Y) (B-inner product)."""
    BY = Y if B is None else B @ Y
    M = X.T @ BY
    return np.linalg.svd(M, compute_uv=False)


def cluster_groups(ev, rel=1e-6):
    groups, cur = [], [0]
    for i in range(1, len(ev)):
        if abs(ev[i] - ev[i - 1]) <= rel * abs(ev[i]):
            cur.append(i)
        else:
            groups.append(cur)
            cur = [i]
    groups.append(cur)
    return groups
