"""GB300 (sm_103a) randomized Block Krylov Iteration and Simultaneous Iteration.

Python face of libbks.so (include/bks.h): Musco & Musco, "Randomized Block Krylov
Methods for Stronger and Faster Approximate Singular Value Decomposition"
(arXiv 1504.05477), Algorithms 1 and 2.  Every function marshals torch tensors
(device memory) and the current CUDA stream into a C-ABI call; the computation runs
in the library's kernels.  There is no CPU fallback: without the CUDA library or a
GPU these functions raise.
"""
from __future__ import annotations

import ctypes

from . import _binding as B
from ._binding import BksError, BksMatrix, BksOpts, BksStats  # noqa: F401

__all__ = ["block_krylov", "simul_iter", "matmul", "orthonormalize", "sym_eig", "gen_pi", "CsrMatrix",
           "gen_pi_host", "Context", "context", "dense_matrix", "BksError", "lib_path"]


def lib_path() -> str:
    return B.lib_path()


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    table = {torch.float64: B.BKS_F64, torch.float32: B.BKS_F32, torch.bfloat16: B.BKS_BF16}
    if t not in table:
        raise TypeError(f"unsupported dtype {t}")
    return table[t]


class Context:
    """One library context (bks_ctx) bound to a CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = B.load()
        ptr = ctypes.c_void_p()
        B.check(self.lib.bks_create(ctypes.byref(ptr), int(device)), None, "bks_create")
        self.ptr = ptr
        self.device = int(device)

    def bind_stream(self):
        torch = _torch()
        s = torch.cuda.current_stream(self.device).cuda_stream
        B.check(self.lib.bks_set_stream(self.ptr, ctypes.c_void_p(s)), self.ptr, "bks_set_stream")

    def set_workspace(self, buf):
        """Give the context a caller-owned device workspace (a torch uint8 tensor)."""
        ptr = ctypes.c_void_p(buf.data_ptr()) if buf is not None else None
        n = buf.numel() if buf is not None else 0
        B.check(self.lib.bks_set_workspace(self.ptr, ptr, n), self.ptr, "bks_set_workspace")
        self._ws = buf

    def close(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            self.lib.bks_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_CTX: dict[int, Context] = {}


def context(device) -> Context:
    torch = _torch()
    dev = torch.device(device)
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    if idx not in _CTX:
        _CTX[idx] = Context(idx)
    ctx = _CTX[idx]
    ctx.bind_stream()
    return ctx


def dense_matrix(a) -> BksMatrix:
    """bks_matrix view of a row-major CUDA tensor (rows contiguous)."""
    if not a.is_cuda or a.dim() != 2 or a.stride(1) != 1:
        raise ValueError("A must be a 2-D CUDA tensor with contiguous rows")
    m = BksMatrix()
    m.kind = B.BKS_DENSE
    m.dtype = _dtype_code(a.dtype)
    m.n, m.d = a.shape
    m.ld = a.stride(0)
    m.vals = a.data_ptr()
    return m


class CsrMatrix:
    """A sparse n x d matrix in CSR form on a CUDA device: row_ptr (int64, n+1), col_idx
    (int32, sorted within rows), vals (float32).  The CSR of A^T is built once by the
    library (bks_csr_transpose) unless transpose=False.  col_mean (d float32) makes every
    product use the implicitly centred A - 1 mu^T."""

    def __init__(self, row_ptr, col_idx, vals, shape, col_mean=None, transpose=True):
        torch = _torch()
        self.row_ptr = row_ptr.to(torch.int64).contiguous()
        self.col_idx = col_idx.to(torch.int32).contiguous()
        self.vals = vals.to(torch.float32).contiguous()
        self.shape = (int(shape[0]), int(shape[1]))
        self.device = self.vals.device
        self.col_mean = col_mean.to(torch.float32).contiguous() if col_mean is not None else None
        self.t = None
        if transpose:
            n, d = self.shape
            nnz = self.vals.numel()
            t_rp = torch.empty(d + 1, dtype=torch.int64, device=self.device)
            t_ci = torch.empty(max(nnz, 1), dtype=torch.int32, device=self.device)
            t_cv = torch.empty(max(nnz, 1), dtype=torch.float32, device=self.device)
            ctx = context(self.device)
            m = self.bks()
            B.check(ctx.lib.bks_csr_transpose(ctx.ptr, ctypes.byref(m), ctypes.c_void_p(t_rp.data_ptr()),
                                              ctypes.c_void_p(t_ci.data_ptr()),
                                              ctypes.c_void_p(t_cv.data_ptr())),
                    ctx.ptr, "bks_csr_transpose")
            self.t = (t_rp, t_ci, t_cv)

    def bks(self) -> BksMatrix:
        m = BksMatrix()
        m.kind = B.BKS_CSR
        m.dtype = B.BKS_F32
        m.n, m.d = self.shape
        m.ld = self.shape[1]
        m.vals = self.vals.data_ptr()
        m.row_ptr = self.row_ptr.data_ptr()
        m.col_idx = self.col_idx.data_ptr()
        m.nnz = self.vals.numel()
        if self.t is not None:
            m.t_row_ptr, m.t_col_idx, m.t_vals = (x.data_ptr() for x in self.t)
        if self.col_mean is not None:
            m.col_mean = self.col_mean.data_ptr()
        return m


def _as_bks(a, precision="auto"):
    """(bks_matrix, device, result dtype) for a dense tensor or a CsrMatrix."""
    torch = _torch()
    if isinstance(a, CsrMatrix):
        return a.bks(), a.device, torch.float32
    return dense_matrix(a), a.device, _out_dtype(a, precision)


def _opts(precision="auto", basis_only=False, sign_fix=True, profile=False, jacobi_tol=0.0,
          jacobi_max_sweeps=40, refine=True, simt=False):
    o = BksOpts()
    B.load().bks_opts_default(ctypes.byref(o))
    o.precision = {"auto": B.PREC_AUTO, "f64": B.PREC_F64, "f32": B.PREC_F32,
                   "bf16": B.PREC_BF16}[precision]
    o.basis_only = int(basis_only)
    o.sign_fix = int(sign_fix)
    o.profile = int(profile)
    o.jacobi_tol = float(jacobi_tol)
    o.jacobi_max_sweeps = int(jacobi_max_sweeps)
    o.refine = int(refine)
    o.product_path = 1 if simt else 0
    return o


def _out_dtype(a, precision):
    torch = _torch()
    if precision == "f64" or (precision == "auto" and a.dtype == torch.float64):
        return torch.float64
    return torch.float32


def _solve(fn_name, a, k, q, seed, pi, want_v, precision, stats, **kw):
    torch = _torch()
    mat, dev, odt = _as_bks(a, precision)
    ctx = context(dev)
    n, d = mat.n, mat.d
    z = torch.empty((n, k), dtype=odt, device=dev)
    sig = torch.empty((k,), dtype=odt, device=dev)
    v = torch.empty((d, k), dtype=odt, device=dev) if want_v else None
    if pi is not None:
        if pi.shape != (d, k) or pi.dtype != odt or not pi.is_contiguous() or pi.device != z.device:
            raise ValueError(f"pi must be a contiguous {d}x{k} {odt} tensor on {z.device}")
    opts = _opts(precision=precision, **kw)
    st = BksStats()
    fn = getattr(ctx.lib, fn_name)
    status = fn(ctx.ptr, ctypes.byref(mat), int(k), int(q), ctypes.c_uint64(seed & (2**64 - 1)),
                ctypes.c_void_p(pi.data_ptr()) if pi is not None else None,
                ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(sig.data_ptr()),
                ctypes.c_void_p(v.data_ptr()) if v is not None else None,
                ctypes.byref(opts), ctypes.byref(st))
    B.check(status, ctx.ptr, fn_name)
    out = (z, sig, v) if want_v else (z, sig)
    return (out + (st.as_dict(),)) if stats else out


def block_krylov(a, k, q, seed=0, pi=None, want_v=False, precision="auto", stats=False, **kw):
    """Algorithm 2 (Block Krylov Iteration) on a CUDA matrix A (n x d).  Returns
    Z (n x k, orthonormal Ritz vectors) and sigma (k Ritz values, descending); with
    want_v also V (d x k); with stats also a dict of bks_stats."""
    return _solve("bks_block_krylov", a, k, q, seed, pi, want_v, precision, stats, **kw)


def simul_iter(a, k, q, seed=0, pi=None, want_v=False, precision="auto", stats=False, **kw):
    """Algorithm 1 (Simultaneous Iteration), same interface as block_krylov."""
    return _solve("bks_simul_iter", a, k, q, seed, pi, want_v, precision, stats, **kw)


def _colmajor(x, pad=1):
    """Column-major copy of a (rows x c) tensor as a (c x ld) array, ld = rows rounded up
    to a multiple of `pad` (torch keeps stride 1 on size-1 dimensions, so .contiguous()
    is not enough).  Returns the (c x rows) view."""
    rows, c = x.shape
    ld = (rows + pad - 1) // pad * pad
    out = _torch().zeros((c, ld), dtype=x.dtype, device=x.device)
    out[:, :rows].copy_(x.t())
    return out[:, :rows]


def matmul(a, x, trans=False, simt=False, exact=False):
    """Y = A X (trans False) or Y = A^T X (trans True) through bks_matmul.  x is a
    (rows x c) CUDA tensor; the result is (rows' x c) in x's dtype.  simt forces the
    CUDA-core kernel; exact asks for the FP32-accurate split product on a BF16 A."""
    torch = _torch()
    mat, dev, _ = _as_bks(a)
    ctx = context(dev)
    xt = _colmajor(x, pad=32)   # 128-byte aligned columns keep the tensor-core path open
    rows_y = mat.d if trans else mat.n
    yt = torch.empty((x.shape[1], (rows_y + 31) // 32 * 32), dtype=x.dtype, device=x.device)[:, :rows_y]
    B.check(ctx.lib.bks_matmul(ctx.ptr, ctypes.byref(mat), int(trans), x.shape[1],
                               ctypes.c_void_p(xt.data_ptr()), xt.stride(0),
                               ctypes.c_void_p(yt.data_ptr()), yt.stride(0),
                               (1 if exact else 0) | (2 if simt else 0)),
            ctx.ptr, "bks_matmul")
    return yt.t()


def orthonormalize(w, qb=None):
    """Project W (len x c) twice against the orthonormal columns of Qb (len x m) and
    orthonormalise it by CholeskyQR2 (bks_orthonormalize).  Returns a new tensor."""
    torch = _torch()
    ctx = context(w.device)
    code = _dtype_code(w.dtype)
    wt = _colmajor(w)
    m = 0 if qb is None else qb.shape[1]
    if m:
        qt = _colmajor(qb)
        if qt.stride(0) != wt.stride(0):
            raise ValueError("Qb and W must have the same length")
        qptr = ctypes.c_void_p(qt.data_ptr())
    else:
        qptr = None
    B.check(ctx.lib.bks_orthonormalize(ctx.ptr, code, w.shape[0], m, w.shape[1], qptr,
                                       wt.stride(0), ctypes.c_void_p(wt.data_ptr()), wt.stride(0)),
            ctx.ptr, "bks_orthonormalize")
    return wt.t()


def sym_eig(m):
    """Eigen-decomposition of a symmetric PSD CUDA matrix by one-sided Jacobi
    (bks_sym_eig): returns (lam descending, U with eigenvectors as columns)."""
    torch = _torch()
    ctx = context(m.device)
    mc = m.contiguous()
    w = mc.shape[0]
    lam = torch.empty((w,), dtype=m.dtype, device=m.device)
    u = torch.empty((w, w), dtype=m.dtype, device=m.device)
    B.check(ctx.lib.bks_sym_eig(ctx.ptr, _dtype_code(m.dtype), w, ctypes.c_void_p(mc.data_ptr()),
                                mc.stride(0), ctypes.c_void_p(lam.data_ptr()),
                                ctypes.c_void_p(u.data_ptr()), u.stride(0)),
            ctx.ptr, "bks_sym_eig")
    return lam, u


def gen_pi(seed, d, k, dtype=None, device="cuda"):
    """Pi (d x k) from the library's SplitMix64 -> Box-Muller generator, on the device."""
    torch = _torch()
    dtype = dtype or torch.float32
    ctx = context(device)
    out = torch.empty((d, k), dtype=dtype, device=device)
    B.check(ctx.lib.bks_gen_pi(ctx.ptr, ctypes.c_uint64(seed), d, k, _dtype_code(dtype),
                               ctypes.c_void_p(out.data_ptr())), ctx.ptr, "bks_gen_pi")
    return out


def gen_pi_host(seed, d, k):
    """Same generator in the library's host code (numpy FP32 array), no GPU needed."""
    import numpy as np
    out = np.empty((d, k), dtype=np.float32)
    B.check(B.load().bks_gen_pi_host(ctypes.c_uint64(seed), d, k,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
            None, "bks_gen_pi_host")
    return out
