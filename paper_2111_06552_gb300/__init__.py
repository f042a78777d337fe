"""Python binding of the GB300 GCG eigensolver library (``libgcge.so``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the shared library, called through its C ABI (``include/gcge.h``).
Functions keep the C names (``gcge_create``, ``gcge_solve``, ...); device
buffers are passed as torch CUDA tensors (or raw integer addresses), host
buffers as numpy arrays.  There is no fallback: if the library or a CUDA
device is missing the calls raise.

Higher-level helpers:
  * ``Solver``    -- owns a handle; ``solve()`` returns (eigenvalues, eigenvectors).
  * ``EigGCG``    -- torch.autograd.Function with the adjoint backward (gradients
                     on the CSR nonzeros of A).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libgcge.so")
_lib = None

GCGE_OK = 0
GCGE_EINVAL = -1
GCGE_ENOMEM = -2
GCGE_ECUDA = -3
GCGE_ENOTCONV = -4
GCGE_EBREAKDOWN = -5
GCGE_ETIMEOUT = -6
GCGE_ENAN = -7
GCGE_ENOTREADY = -8
GCGE_FP64 = 0
GCGE_MIXED = 1
GCGE_PRECOND_NONE = 0
GCGE_PRECOND_JACOBI = 1
GCGE_ORTH_ALG3 = 0
GCGE_ORTH_ALG2 = 1
KERNEL_CLASSES = ("spmm", "gram", "vc", "syev", "cgvec", "other", "spmm64", "gram64", "vc64",
                  "gram64tc", "vc64tc")


class GcgeError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().gcge_error_string(status).decode()
        detail = lib().gcge_last_error_message().decode()
        super().__init__(f"{where}: status {status} ({msg}); {detail}")
        self.status = status


class gcge_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("on_device", C.c_int)]


class gcge_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("cg_max_iter", C.c_int), ("cg_rtol", C.c_double),
                ("use_shift", C.c_int), ("orth_leaf", C.c_int), ("moving", C.c_int),
                ("size_x", C.c_int), ("max_iter", C.c_int), ("seed", C.c_uint64),
                ("initial_block", C.c_void_p), ("mixed_switch_tol", C.c_double),
                ("verbose", C.c_int), ("checks", C.c_int), ("profile", C.c_int),
                ("mixed_bs2", C.c_int), ("orth", C.c_int), ("precond", C.c_int),
                ("fp64_emulation", C.c_int), ("max_proj_dim", C.c_int)]


class gcge_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("iterations_fp32", C.c_int), ("nconv", C.c_int),
                ("cg_steps", C.c_int64), ("moves", C.c_int), ("ms_total", C.c_double),
                ("ms_step", C.c_double * 7), ("ms_syev", C.c_double),
                ("max_orth_err", C.c_double), ("max_abar_err", C.c_double),
                ("kernel_launches", C.c_int64), ("prof_ms", C.c_double * 12),
                ("prof_calls", C.c_int64 * 12), ("prof_bytes", C.c_double * 12),
                ("prof_flops", C.c_double * 12), ("refills", C.c_int)]


_P = C.c_void_p
_I64 = C.c_int64
_I = C.c_int
_D = C.c_double
_F = C.c_float

_SIGS = {
    "gcge_options_default": (_I, [C.POINTER(gcge_options)]),
    "gcge_create": (_I, [C.POINTER(gcge_csr), C.POINTER(gcge_csr), _I, _I, _D,
                         C.POINTER(gcge_options), _P, C.POINTER(_P)]),
    "gcge_solve": (_I, [_P]),
    "gcge_eigenpairs": (_I, [_P, _P, _P, _I64, _I, C.POINTER(_I)]),
    "gcge_stats_get": (_I, [_P, C.POINTER(gcge_stats)]),
    "gcge_eig_grad": (_I, [_P, _I, _P, _P, _I64, _P, _D]),
    "gcge_error_string": (C.c_char_p, [_I]),
    "gcge_last_error_message": (C.c_char_p, []),
    "gcge_destroy": (None, [_P]),
    "gcge_spmm_f64": (_I, [_I64, _P, _P, _P, _I, _D, _P, _I64, _D, _P, _I64, _P]),
    "gcge_spmm_f32": (_I, [_I64, _P, _P, _P, _I, _F, _P, _I64, _F, _P, _I64, _P]),
    "gcge_gram_f64": (_I, [_I64, _I, _I, _D, _P, _I64, _P, _I64, _D, _P, _I64, _P]),
    "gcge_gram_f32": (_I, [_I64, _I, _I, _D, _P, _I64, _P, _I64, _D, _P, _I64, _I, _P]),
    "gcge_vc_f64": (_I, [_I64, _I, _I, _D, _P, _I64, _P, _I64, _D, _P, _I64, _P]),
    "gcge_vc_f32": (_I, [_I64, _I, _I, _D, _P, _I64, _P, _I64, _D, _P, _I64, _I, _P]),
    "gcge_syev": (_I, [_I, _P, _I64, _P, _P, _I64, C.POINTER(_I), _P]),
    "gcge_block_cg_f64": (_I, [_I64, _P, _P, _P, _I, _P, _I64, _P, _I64, _I, _D, _I, _P, _P]),
    "gcge_block_cg_f32": (_I, [_I64, _P, _P, _P, _I, _P, _I64, _P, _I64, _I, _D, _I, _P, _P]),
    "gcge_borth_f64": (_I, [_I64, _P, _P, _P, _P, _I64, _I, _P, _I64, _I, _I, _I, C.POINTER(_I),
                            _P]),
    "gcge_random_block_f64": (_I, [_I64, _I, C.c_uint64, _P, _I64, _P]),
    "gcge_tc_status": (_I, [_P]),
    "gcge_gram_f64_noalloc": (_I, [_I64, _I, _I, _D, _P, _I64, _P, _I64, _D, _P, _I64, _P]),
    "gcge_gram_f64_tc": (_I, [_I64, _I, _I, _D, _P, _I64, _P, _I64, _D, _P, _I64, _P]),
    "gcge_vc_f64_tc": (_I, [_I64, _I, _I, _D, _P, _I64, _P, _I64, _D, _P, _I64, _P]),
}
GCGE_GRAM_NOALLOC_MAX_DOUBLES = 2 * 1024 * 1024


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load ``libgcge.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: run paper_2111_06552_gb300.build.build()")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _addr(x):
    """Device/host address of a torch tensor, numpy array, or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(status: int, where: str) -> int:
    if status != GCGE_OK:
        raise GcgeError(status, where)
    return status


# ------------------------------------------------------------------ step-level calls
def gcge_spmm_f64(n, row_ptr, col_idx, val, k, alpha, X, ldx, beta, Y, ldy, stream=None):
    return _check(lib().gcge_spmm_f64(n, _addr(row_ptr), _addr(col_idx), _addr(val), k, alpha,
                                      _addr(X), ldx, beta, _addr(Y), ldy, _stream(stream)),
                  "gcge_spmm_f64")


def gcge_spmm_f32(n, row_ptr, col_idx, val, k, alpha, X, ldx, beta, Y, ldy, stream=None):
    return _check(lib().gcge_spmm_f32(n, _addr(row_ptr), _addr(col_idx), _addr(val), k, alpha,
                                      _addr(X), ldx, beta, _addr(Y), ldy, _stream(stream)),
                  "gcge_spmm_f32")


def gcge_gram_f64(n, m, k, alpha, X, ldx, Y, ldy, beta, Cm, ldc, stream=None):
    return _check(lib().gcge_gram_f64(n, m, k, alpha, _addr(X), ldx, _addr(Y), ldy, beta,
                                      _addr(Cm), ldc, _stream(stream)), "gcge_gram_f64")


def gcge_gram_f64_noalloc(n, m, k, alpha, X, ldx, Y, ldy, beta, Cm, ldc, stream=None):
    """gcge_gram_f64 without device allocation (static library scratch; see gcge.h)."""
    return _check(lib().gcge_gram_f64_noalloc(n, m, k, alpha, _addr(X), ldx, _addr(Y), ldy, beta,
                                              _addr(Cm), ldc, _stream(stream)),
                  "gcge_gram_f64_noalloc")


def gcge_gram_f64_tc(n, m, k, alpha, X, ldx, Y, ldy, beta, Cm, ldc, stream=None):
    _check(lib().gcge_gram_f64_tc(n, m, k, alpha, _addr(X), ldx, _addr(Y), ldy, beta, _addr(Cm),
                                  ldc, _stream(stream)), "gcge_gram_f64_tc")


def gcge_vc_f64_tc(n, d, q, alpha, V, ldv, Cm, ldc, beta, Y, ldy, stream=None):
    _check(lib().gcge_vc_f64_tc(n, d, q, alpha, _addr(V), ldv, _addr(Cm), ldc, beta, _addr(Y),
                                ldy, _stream(stream)), "gcge_vc_f64_tc")


def gcge_gram_f32(n, m, k, alpha, X, ldx, Y, ldy, beta, Cm, ldc, tc=1, stream=None):
    return _check(lib().gcge_gram_f32(n, m, k, alpha, _addr(X), ldx, _addr(Y), ldy, beta,
                                      _addr(Cm), ldc, tc, _stream(stream)), "gcge_gram_f32")


def gcge_vc_f64(n, d, q, alpha, V, ldv, Cm, ldc, beta, Y, ldy, stream=None):
    return _check(lib().gcge_vc_f64(n, d, q, alpha, _addr(V), ldv, _addr(Cm), ldc, beta,
                                    _addr(Y), ldy, _stream(stream)), "gcge_vc_f64")


def gcge_vc_f32(n, d, q, alpha, V, ldv, Cm, ldc, beta, Y, ldy, tc=1, stream=None):
    return _check(lib().gcge_vc_f32(n, d, q, alpha, _addr(V), ldv, _addr(Cm), ldc, beta,
                                    _addr(Y), ldy, tc, _stream(stream)), "gcge_vc_f32")


def gcge_syev(d, A, lda, w, Q, ldq, stream=None):
    sweeps = C.c_int(0)
    _check(lib().gcge_syev(d, _addr(A), lda, _addr(w), _addr(Q), ldq, C.byref(sweeps),
                           _stream(stream)), "gcge_syev")
    return sweeps.value


def gcge_block_cg_f64(n, row_ptr, col_idx, S, k, Bm, ldb, X, ldx, max_iter, rtol, precond=0,
                      stream=None):
    it = np.zeros(k, dtype=np.int32)
    _check(lib().gcge_block_cg_f64(n, _addr(row_ptr), _addr(col_idx), _addr(S), k, _addr(Bm), ldb,
                                   _addr(X), ldx, max_iter, rtol, precond, it.ctypes.data,
                                   _stream(stream)), "gcge_block_cg_f64")
    return it


def gcge_block_cg_f32(n, row_ptr, col_idx, S, k, Bm, ldb, X, ldx, max_iter, rtol, precond=0,
                      stream=None):
    it = np.zeros(k, dtype=np.int32)
    _check(lib().gcge_block_cg_f32(n, _addr(row_ptr), _addr(col_idx), _addr(S), k, _addr(Bm), ldb,
                                   _addr(X), ldx, max_iter, rtol, precond, it.ctypes.data,
                                   _stream(stream)), "gcge_block_cg_f32")
    return it


def gcge_borth_f64(n, Brp, Bci, Bval, Q, ldq, q, W, ldw, m, leaf=16, orth=GCGE_ORTH_ALG3,
                   stream=None):
    out = C.c_int(0)
    _check(lib().gcge_borth_f64(n, _addr(Brp), _addr(Bci), _addr(Bval), _addr(Q), ldq, q,
                                _addr(W), ldw, m, leaf, orth, C.byref(out), _stream(stream)),
           "gcge_borth_f64")
    return out.value


def gcge_tc_status(stream=None):
    """GCGE_OK, or raises on GCGE_ETIMEOUT (a tensor-core kernel's bounded wait ran out)."""
    return _check(lib().gcge_tc_status(_stream(stream)), "gcge_tc_status")


def gcge_random_block_f64(n, k, seed, X, ld, stream=None):
    return _check(lib().gcge_random_block_f64(n, k, seed, _addr(X), ld, _stream(stream)),
                  "gcge_random_block_f64")


def gcge_options_default() -> gcge_options:
    o = gcge_options()
    _check(lib().gcge_options_default(C.byref(o)), "gcge_options_default")
    return o


# ------------------------------------------------------------------ handle-level
def _csr_struct(mat, keep):
    """gcge_csr for a scipy CSR matrix (host) or a (row_ptr, col_idx, val) tensor triple."""
    if mat is None:
        return None
    if isinstance(mat, tuple):
        rp, ci, val = mat
        n = rp.numel() - 1
        on_dev = 1 if rp.is_cuda else 0
        keep.extend([rp, ci, val])
        return gcge_csr(n, ci.numel(), _addr(rp), _addr(ci), _addr(val), on_dev)
    rp = np.ascontiguousarray(mat.indptr, dtype=np.int32)
    ci = np.ascontiguousarray(mat.indices, dtype=np.int32)
    val = np.ascontiguousarray(mat.data, dtype=np.float64)
    keep.extend([rp, ci, val])
    return gcge_csr(mat.shape[0], mat.nnz, rp.ctypes.data, ci.ctypes.data, val.ctypes.data, 0)


def gcge_create(A, B, nev, block_size, tol, options=None, stream=None):
    keep = []
    a = _csr_struct(A, keep)
    b = _csr_struct(B, keep)
    h = C.c_void_p()
    _check(lib().gcge_create(C.byref(a), C.byref(b) if b is not None else None, nev, block_size,
                             tol, C.byref(options) if options is not None else None,
                             _stream(stream), C.byref(h)), "gcge_create")
    return h


def gcge_solve(h):
    s = lib().gcge_solve(h)
    if s not in (GCGE_OK, GCGE_ENOTCONV):
        _check(s, "gcge_solve")
    return s


def gcge_eigenpairs(h, nev, n, evecs=None, on_device=False):
    """Fill and return (evals (numpy), nconv); evecs is an n x nev column-major buffer."""
    ev = np.zeros(nev, dtype=np.float64)
    nc = C.c_int(0)
    ldv = n
    _check(lib().gcge_eigenpairs(h, ev.ctypes.data, _addr(evecs), ldv, 1 if on_device else 0,
                                 C.byref(nc)), "gcge_eigenpairs")
    return ev, nc.value


def gcge_stats_get(h) -> gcge_stats:
    st = gcge_stats()
    _check(lib().gcge_stats_get(h, C.byref(st)), "gcge_stats_get")
    return st


def gcge_eig_grad(h, k, w_lambda, d_gx, ldg, d_dA, adj_tol=1e-12):
    w = None if w_lambda is None else np.ascontiguousarray(w_lambda, dtype=np.float64)
    return _check(lib().gcge_eig_grad(h, k, _addr(w), _addr(d_gx), ldg, _addr(d_dA), adj_tol),
                  "gcge_eig_grad")


def gcge_destroy(h):
    lib().gcge_destroy(h)


def stats_dict(st: gcge_stats) -> dict:
    return {"iterations": st.iterations, "iterations_fp32": st.iterations_fp32,
            "nconv": st.nconv, "cg_steps": st.cg_steps, "moves": st.moves,
            "refills": st.refills,
            "ms_total": st.ms_total, "ms_step": list(st.ms_step), "ms_syev": st.ms_syev,
            "max_orth_err": st.max_orth_err, "max_abar_err": st.max_abar_err,
            "kernel_launches": st.kernel_launches,
            "prof": {name: {"ms": st.prof_ms[i], "calls": st.prof_calls[i],
                            "bytes": st.prof_bytes[i], "flops": st.prof_flops[i]}
                     for i, name in enumerate(KERNEL_CLASSES)}}


class Solver:
    """Owns one gcge handle for a pencil (A, B); ``solve()`` returns eigenpairs.

    A, B: scipy CSR (host) or (row_ptr, col_idx, val) torch tensors; B None = identity.
    """

    def __init__(self, A, B, nev, block_size, tol=1e-8, precision=GCGE_FP64, stream=None,
                 **opts):
        self.n = A.shape[0] if not isinstance(A, tuple) else A[0].numel() - 1
        self.nev = nev
        self.opt = gcge_options_default()
        self.opt.precision = precision
        self._init_block = None
        for k, v in opts.items():
            if k == "initial_block":
                self._init_block = np.ascontiguousarray(v, dtype=np.float64)
                self.opt.initial_block = self._init_block.ctypes.data
            else:
                setattr(self.opt, k, v)
        self.h = gcge_create(A, B, nev, block_size, tol, self.opt, stream)
        self.status = None

    def solve(self, evecs_device=None):
        """Run the solve; returns (evals numpy, evecs) with evecs an n x nev column-major
        buffer: the given device tensor, or a new host numpy array."""
        self.status = gcge_solve(self.h)
        if evecs_device is not None:
            ev, self.nconv = gcge_eigenpairs(self.h, self.nev, self.n, evecs_device, True)
            return ev, evecs_device
        out = np.zeros((self.nev, self.n), dtype=np.float64)   # column-major n x nev
        ev, self.nconv = gcge_eigenpairs(self.h, self.nev, self.n, out, False)
        return ev, out.T

    def stats(self) -> dict:
        return stats_dict(gcge_stats_get(self.h))

    def close(self):
        if self.h is not None:
            gcge_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build():
    from .build import build as _b
    return _b()


# ------------------------------------------------------------------ autograd
def _torch():
    import torch
    return torch


class _CsrDev:
    """A CSR matrix held as device tensors (row_ptr, col_idx, values)."""

    def __init__(self, M, device="cuda"):
        torch = _torch()
        self.n_rows = M.shape[0]
        self.rp = torch.tensor(np.asarray(M.indptr, dtype=np.int32), device=device)
        self.ci = torch.tensor(np.asarray(M.indices, dtype=np.int32), device=device)
        self.val = torch.tensor(np.asarray(M.data, dtype=np.float64), device=device)


class CellMap:
    """Linear map c -> A(c).data given by a sparse Jacobian J (nnz x cells), applied and
    transposed with the library's SpMM (k = 1)."""

    def __init__(self, J):
        self.J = _CsrDev(J)
        self.JT = _CsrDev(J.T.tocsr())
        self.nnz = J.shape[0]
        self.ncell = J.shape[1]

    def apply(self, c):
        torch = _torch()
        out = torch.empty(self.nnz, dtype=torch.float64, device=c.device)
        gcge_spmm_f64(self.nnz, self.J.rp, self.J.ci, self.J.val, 1, 1.0, c.contiguous(), 1, 0.0,
                      out, 1)
        return out

    def apply_t(self, g):
        torch = _torch()
        out = torch.empty(self.ncell, dtype=torch.float64, device=g.device)
        gcge_spmm_f64(self.ncell, self.JT.rp, self.JT.ci, self.JT.val, 1, 1.0, g.contiguous(), 1,
                      0.0, out, 1)
        return out


def cells_to_values(c, cmap: CellMap):
    """Differentiable A(c).data = J c (backward: J^T g on the library's SpMM)."""
    torch = _torch()

    class _F(torch.autograd.Function):
        @staticmethod
        def forward(ctx, cc):
            return cmap.apply(cc)

        @staticmethod
        def backward(ctx, g):
            return cmap.apply_t(g)

    return _F.apply(c)


class EigGCG:
    """Differentiable smallest-nev eigenpairs of A(a_vals) x = lambda B x.

    ``EigGCG.apply(a_vals, pattern, B, nev, bs, tol, adj_tol, opts)`` returns
    (eigenvalues (nev,), eigenvectors (n, nev)) as device tensors; the backward pass
    calls gcge_eig_grad (adjoint kernel) and returns dL/da_vals on A's CSR pattern.
    pattern = (row_ptr, col_idx) device int32 tensors; B a scipy CSR or None.
    """

    @staticmethod
    def apply(a_vals, pattern, B, nev, bs, tol=1e-8, adj_tol=1e-12, opts=None):
        torch = _torch()
        rp, ci = pattern
        opts = dict(opts or {})

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, av):
                solver = Solver((rp, ci, av.detach().contiguous()), B, nev, bs, tol, **opts)
                n = solver.n
                ev_buf = torch.empty((nev, n), dtype=torch.float64, device=av.device)
                ev, _ = solver.solve(evecs_device=ev_buf)
                ctx.solver = solver
                ctx.n = n
                return (torch.tensor(ev, dtype=torch.float64, device=av.device),
                        ev_buf.t())

            @staticmethod
            def backward(ctx, g_ev, g_x):
                solver = ctx.solver
                w = (g_ev.detach().cpu().numpy().astype(np.float64) if g_ev is not None
                     else np.zeros(nev))
                gx = None
                if g_x is not None:
                    gx = g_x.detach().to(torch.float64).contiguous()
                out = torch.empty(ci.numel(), dtype=torch.float64, device=rp.device)
                gcge_eig_grad(solver.h, nev, w, gx, nev, out, adj_tol)
                return out

        return _F.apply(a_vals)
