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

__all__ = ["block_krylov", "block_krylov_adaptive", "block_lanczos", "simul_iter", "matmul", "orthonormalize", "sym_eig", "gen_pi", "CsrMatrix",
           "ritz_triplets", "low_rank", "backward", "rand_svd", "krylov_width", "block_krylov_batched",
           "ritz_triplets_batched", "backward_batched", "rand_svd_batched", "batch_budget", "batched_autotune",
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
          jacobi_max_sweeps=40, refine=True, simt=False, rr_mode="auto", eig_mode="auto", block_p=0,
          eig_f64=False, max_sms=0):
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
    o.rr_mode = {"auto": 0, "qr": 1, "gram": 2}[rr_mode]
    o.eig_mode = {"auto": 0, "jacobi": 1}[eig_mode]
    o.block_p = int(block_p)
    o.eig_f64 = int(eig_f64)
    o.max_sms = int(max_sms)
    return o


def _out_dtype(a, precision):
    torch = _torch()
    if precision == "f64" or (precision == "auto" and a.dtype == torch.float64):
        return torch.float64
    return torch.float32


def _solve(fn_name, a, k, q, seed, pi, want_v, precision, stats, _tol=None, _reorth=None, **kw):
    torch = _torch()
    mat, dev, odt = _as_bks(a, precision)
    ctx = context(dev)
    n, d = mat.n, mat.d
    z = torch.empty((n, k), dtype=odt, device=dev)
    sig = torch.empty((k,), dtype=odt, device=dev)
    v = torch.empty((d, k), dtype=odt, device=dev) if want_v else None
    if pi is not None:
        pc = kw.get("block_p") or k
        if pi.shape != (d, pc) or pi.dtype != odt or not pi.is_contiguous() or pi.device != z.device:
            raise ValueError(f"pi must be a contiguous {d}x{pc} {odt} tensor on {z.device}")
    opts = _opts(precision=precision, **kw)
    st = BksStats()
    fn = getattr(ctx.lib, fn_name)
    head = (ctx.ptr, ctypes.byref(mat), int(k), int(q))
    if _tol is not None:
        head = head + (ctypes.c_double(_tol),)
    if _reorth is not None:
        head = head + (int(_reorth),)
    status = fn(*head, ctypes.c_uint64(seed & (2**64 - 1)),
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
    want_v also V (d x k); with stats also a dict of bks_stats.  block_p = p > k runs the
    iteration with p columns in Pi and in every block (Sec. 8); pi is then d x p."""
    return _solve("bks_block_krylov", a, k, q, seed, pi, want_v, precision, stats, **kw)


def block_krylov_adaptive(a, k, q_max, tol, seed=0, pi=None, want_v=False, precision="auto", stats=False, **kw):
    """Algorithm 2 with q chosen on the fly (bks_block_krylov_adaptive): stops once none of
    the k leading Ritz values moves by more than tol (relative) between iterations, at most
    q_max iterations; stats["q_eff"] reports the iterations run."""
    return _solve("bks_block_krylov_adaptive", a, k, q_max, seed, pi, want_v, precision, stats,
                  _tol=float(tol), **kw)


def block_lanczos(a, k, q, seed=0, pi=None, reorth="full", want_v=False, precision="auto", stats=False, **kw):
    """Block Lanczos (Sec. 4; bks_block_lanczos): the Krylov space of Algorithm 2 built by
    the three-term block recurrence, with Rayleigh-Ritz on the block-tridiagonal
    T = Q^T A A^T Q.  reorth: "full" (twice against every earlier block), "local" (against
    the two previous blocks) or "none".  Same interface and results as block_krylov."""
    if reorth not in B.REORTH:
        raise ValueError("reorth must be 'full', 'local' or 'none'")
    return _solve("bks_block_lanczos", a, k, q, seed, pi, want_v, precision, stats,
                  _reorth=B.REORTH[reorth], **kw)


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


# ---------------------------------------------------------------------- differentiation
def krylov_width(n, d, k, q, method="bki"):
    """Number of Ritz triplets of a solve: k(q_eff + 1) for Block Krylov, k for SI."""
    return int(B.load().bks_krylov_width(int(n), int(d), int(k), int(q), 0 if method == "bki" else 1))


def ritz_triplets(a, k, q, seed=0, pi=None, method="bki", precision="auto", **kw):
    """All w Ritz triplets of a solve (bks_ritz_triplets): U (n x w), sigma (w), V (d x w);
    the first k are the solve's Z, Sigma_k and V_k."""
    torch = _torch()
    mat, dev, odt = _as_bks(a, precision)
    ctx = context(dev)
    n, d = mat.n, mat.d
    w = krylov_width(n, d, k, q, method)
    if w < 1:
        raise ValueError("bad sizes")
    u = torch.empty((n, w), dtype=odt, device=dev)
    s = torch.empty((w,), dtype=odt, device=dev)
    v = torch.empty((d, w), dtype=odt, device=dev)
    if pi is not None and (pi.shape != (d, k) or pi.dtype != odt or not pi.is_contiguous()):
        raise ValueError(f"pi must be a contiguous {d}x{k} {odt} tensor")
    opts = _opts(precision=precision, **kw)
    st = BksStats()
    status = ctx.lib.bks_ritz_triplets(ctx.ptr, ctypes.byref(mat), int(k), int(q),
                                       ctypes.c_uint64(seed & (2**64 - 1)),
                                       ctypes.c_void_p(pi.data_ptr()) if pi is not None else None,
                                       0 if method == "bki" else 1, ctypes.c_void_p(u.data_ptr()),
                                       ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                       ctypes.byref(opts), ctypes.byref(st))
    B.check(status, ctx.ptr, "bks_ritz_triplets")
    return u, s, v


def low_rank(u, s, v, r=None):
    """U_r diag(s_r) V_r^T (bks_low_rank) for row-major U (n x w) and V (d x w)."""
    torch = _torch()
    r = s.shape[0] if r is None else int(r)
    u, s, v = u.contiguous(), s.contiguous(), v.contiguous()
    ctx = context(u.device)
    out = torch.empty((u.shape[0], v.shape[0]), dtype=u.dtype, device=u.device)
    B.check(ctx.lib.bks_low_rank(ctx.ptr, _dtype_code(u.dtype), u.shape[0], v.shape[0], r,
                                 ctypes.c_void_p(u.data_ptr()), u.stride(0), ctypes.c_void_p(s.data_ptr()),
                                 ctypes.c_void_p(v.data_ptr()), v.stride(0), ctypes.c_void_p(out.data_ptr())),
            ctx.ptr, "bks_low_rank")
    return out


def backward(u, s, v, k, g_sigma=None, g_ak=None, gap_tau=0.0):
    """dL/dA from the Ritz triplets and the upstream gradients of Sigma_k and A_k
    (bks_backward)."""
    torch = _torch()
    u, s, v = u.contiguous(), s.contiguous(), v.contiguous()
    n, w = u.shape
    d = v.shape[0]
    ctx = context(u.device)
    da = torch.empty((n, d), dtype=u.dtype, device=u.device)
    gs = g_sigma.contiguous().to(u.dtype) if g_sigma is not None else None
    ga = g_ak.contiguous().to(u.dtype) if g_ak is not None else None
    B.check(ctx.lib.bks_backward(ctx.ptr, _dtype_code(u.dtype), n, d, int(k), w,
                                 ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(s.data_ptr()),
                                 ctypes.c_void_p(v.data_ptr()),
                                 ctypes.c_void_p(gs.data_ptr()) if gs is not None else None,
                                 ctypes.c_void_p(ga.data_ptr()) if ga is not None else None,
                                 ctypes.c_void_p(da.data_ptr()), float(gap_tau)),
            ctx.ptr, "bks_backward")
    return da


def _autograd_function():
    torch = _torch()

    class RandSVD(torch.autograd.Function):
        """(Sigma_k, A_k = Z Z^T A) of a randomized solve, differentiable in A.  The backward
        is one bks_backward call on the Ritz triplets (not an unrolling of the iterations).
        The triplets are saved by the forward, or (recompute) rebuilt in the backward by the
        same deterministic solve, which then holds only A and Pi."""

        @staticmethod
        def forward(ctx, a, k, q, seed, pi, method, precision, gap_tau, recompute, max_sms):
            u, s, v = ritz_triplets(a.detach(), k, q, seed=seed, pi=pi, method=method, precision=precision,
                                    max_sms=max_sms)
            if recompute:
                if pi is not None:
                    ctx.save_for_backward(a, pi)
                else:
                    ctx.save_for_backward(a)
            else:
                ctx.save_for_backward(u, s, v)
            ctx.k, ctx.q, ctx.seed, ctx.method, ctx.precision = k, q, seed, method, precision
            ctx.gap_tau, ctx.in_dtype, ctx.recompute, ctx.max_sms = gap_tau, a.dtype, recompute, max_sms
            return s[:k].clone(), low_rank(u, s, v, k)

        @staticmethod
        def backward(ctx, g_sigma, g_ak):
            if ctx.recompute:
                saved = ctx.saved_tensors
                a, pi = saved[0], (saved[1] if len(saved) > 1 else None)
                u, s, v = ritz_triplets(a.detach(), ctx.k, ctx.q, seed=ctx.seed, pi=pi, method=ctx.method,
                                        precision=ctx.precision, max_sms=ctx.max_sms)
            else:
                u, s, v = ctx.saved_tensors
            da = backward(u, s, v, ctx.k, g_sigma, g_ak, ctx.gap_tau)
            return da.to(ctx.in_dtype), None, None, None, None, None, None, None, None, None

    class RandSVDBatched(torch.autograd.Function):
        """rand_svd on a list of matrices: one batched triplets call forward, one batched
        backward call (bks_ritz_triplets_batched, bks_backward_batched)."""

        @staticmethod
        def forward(ctx, k, q, seeds, pis, method, precision, gap_tau, recompute, max_sms, *mats):
            trips = ritz_triplets_batched([m.detach() for m in mats], k, q, seeds=seeds, pis=pis, method=method,
                                          precision=precision, max_sms=max_sms)
            ctx.k, ctx.q, ctx.seeds, ctx.pis, ctx.method, ctx.max_sms = k, q, seeds, pis, method, max_sms
            ctx.precision, ctx.gap_tau, ctx.recompute = precision, gap_tau, recompute
            ctx.in_dtypes = [m.dtype for m in mats]
            if recompute:
                ctx.save_for_backward(*mats)
            else:
                ctx.save_for_backward(*[x for t in trips for x in t])
            out = []
            for u, s, v in trips:
                out += [s[:k].clone(), low_rank(u, s, v, k)]
            return tuple(out)

        @staticmethod
        def backward(ctx, *grads):
            saved = ctx.saved_tensors
            if ctx.recompute:
                trips = ritz_triplets_batched([m.detach() for m in saved], ctx.k, ctx.q, seeds=ctx.seeds,
                                              pis=ctx.pis, method=ctx.method, precision=ctx.precision,
                                              max_sms=ctx.max_sms)
            else:
                trips = [tuple(saved[3 * i:3 * i + 3]) for i in range(len(saved) // 3)]
            das = backward_batched(trips, ctx.k, list(grads[0::2]), list(grads[1::2]), ctx.gap_tau)
            return (None,) * 9 + tuple(da.to(dt) for da, dt in zip(das, ctx.in_dtypes))

    return RandSVD, RandSVDBatched


_RANDSVD = None


def rand_svd(a, k, q, seed=0, pi=None, method="bki", precision="auto", gap_tau=0.0, recompute=False,
             max_sms=0):
    """Differentiable (Sigma_k, A_k) of Block Krylov (method "bki") or Simultaneous
    Iteration ("si") on a dense CUDA matrix.  recompute=True keeps no Ritz triplets between
    forward and backward (only A and Pi) and rebuilds them in the backward; the gradient is
    bit-identical, since the solve is deterministic."""
    global _RANDSVD
    if _RANDSVD is None:
        _RANDSVD = _autograd_function()
    return _RANDSVD[0].apply(a, k, q, seed, pi, method, precision, gap_tau, bool(recompute), int(max_sms))


def rand_svd_batched(mats, k, q, seeds=None, pis=None, method="bki", precision="auto", gap_tau=0.0,
                     recompute=False, max_sms=0):
    """rand_svd on a list of dense CUDA matrices of any shapes, forward and backward each in
    one batched call.  Returns [(Sigma_k, A_k), ...], differentiable in every matrix."""
    global _RANDSVD
    if _RANDSVD is None:
        _RANDSVD = _autograd_function()
    if len(mats) == 0:
        return []
    flat = _RANDSVD[1].apply(k, q, seeds, pis, method, precision, gap_tau, bool(recompute), int(max_sms), *mats)
    return [(flat[2 * i], flat[2 * i + 1]) for i in range(len(mats))]


def batch_budget(mats, k, q, method="bki"):
    """SMs per solve a batched call with max_sms = 0 uses for this batch (bks_batch_budget): the
    budget batched_autotune cached for its signature, else an eighth of the GPU.  A single call
    with max_sms set to it reproduces a batch member bit for bit."""
    b = len(mats)
    arr = (BksMatrix * b)()
    dev = None
    for i, a in enumerate(mats):
        m, dv, _ = _as_bks(a)
        dev = dv if dev is None else dev
        arr[i] = m
    ctx = context(dev)
    return int(ctx.lib.bks_batch_budget(ctx.ptr, b, arr, int(k), int(q), 0 if method == "bki" else 1))


def batched_autotune(mats, k, q, seeds=None, want_v=False, precision="auto", **kw):
    """Times the batch at each candidate SM budget (bks_batched_autotune), caches the fastest for
    batches of this signature and returns (results, budget, ms per batch)."""
    torch = _torch()
    b = len(mats)
    arr = (BksMatrix * b)()
    zp, sp, vp = ((ctypes.c_void_p * b)() for _ in range(3))
    outs, dev = [], None
    for i, a in enumerate(mats):
        m, dv, odt = _as_bks(a, precision)
        dev = dv if dev is None else dev
        arr[i] = m
        z = torch.empty((m.n, k), dtype=odt, device=dv)
        s = torch.empty((k,), dtype=odt, device=dv)
        v = torch.empty((m.d, k), dtype=odt, device=dv) if want_v else None
        zp[i], sp[i] = z.data_ptr(), s.data_ptr()
        if v is not None:
            vp[i] = v.data_ptr()
        outs.append((z, s, v) if want_v else (z, s))
    ctx = context(dev)
    seeds_arr = (ctypes.c_uint64 * b)(*[int(x) & (2**64 - 1) for x in (seeds if seeds is not None else range(b))])
    opts = _opts(precision=precision, **kw)
    best, ms = ctypes.c_int(0), ctypes.c_float(0.0)
    B.check(ctx.lib.bks_batched_autotune(ctx.ptr, b, arr, int(k), int(q), ctypes.cast(seeds_arr, ctypes.c_void_p), None,
                                         ctypes.cast(zp, ctypes.c_void_p), ctypes.cast(sp, ctypes.c_void_p),
                                         ctypes.cast(vp, ctypes.c_void_p) if want_v else None, ctypes.byref(opts),
                                         ctypes.byref(best), ctypes.byref(ms)),
            ctx.ptr, "bks_batched_autotune")
    return outs, best.value, ms.value


def ritz_triplets_batched(mats, k, q, seeds=None, pis=None, method="bki", precision="auto", **kw):
    """ritz_triplets on a list of dense CUDA matrices (or CsrMatrix) in one call
    (bks_ritz_triplets_batched): a list of (U_i, sigma_i, V_i)."""
    torch = _torch()
    b = len(mats)
    if b == 0:
        return []
    arr = (BksMatrix * b)()
    up, sp, vp, pp = ((ctypes.c_void_p * b)() for _ in range(4))
    outs, dev = [], None
    for i, a in enumerate(mats):
        m, dv, odt = _as_bks(a, precision)
        dev = dv if dev is None else dev
        arr[i] = m
        w = krylov_width(m.n, m.d, k, q, method)
        if w < 1:
            raise ValueError(f"bad sizes for matrix {i}")
        u = torch.empty((m.n, w), dtype=odt, device=dv)
        s = torch.empty((w,), dtype=odt, device=dv)
        v = torch.empty((m.d, w), dtype=odt, device=dv)
        up[i], sp[i], vp[i] = u.data_ptr(), s.data_ptr(), v.data_ptr()
        if pis is not None and pis[i] is not None:
            p = pis[i]
            if p.shape != (m.d, k) or p.dtype != odt or not p.is_contiguous():
                raise ValueError(f"pis[{i}] must be a contiguous {m.d}x{k} {odt} tensor")
            pp[i] = p.data_ptr()
        outs.append((u, s, v))
    ctx = context(dev)
    seeds_arr = (ctypes.c_uint64 * b)(*[int(x) & (2**64 - 1) for x in (seeds if seeds is not None else range(b))])
    statuses = (ctypes.c_int32 * b)()
    opts = _opts(precision=precision, **kw)
    status = ctx.lib.bks_ritz_triplets_batched(ctx.ptr, b, arr, int(k), int(q), ctypes.cast(seeds_arr, ctypes.c_void_p),
                                               ctypes.cast(pp, ctypes.c_void_p) if pis is not None else None,
                                               0 if method == "bki" else 1, ctypes.cast(up, ctypes.c_void_p),
                                               ctypes.cast(sp, ctypes.c_void_p), ctypes.cast(vp, ctypes.c_void_p),
                                               ctypes.byref(opts), ctypes.cast(statuses, ctypes.c_void_p))
    B.check(status, ctx.ptr, "bks_ritz_triplets_batched")
    return outs


def backward_batched(triplets, k, g_sigmas=None, g_aks=None, gap_tau=0.0):
    """backward for a list of Ritz triplets (bks_backward_batched).  g_sigmas / g_aks: lists
    (entries may be None) or None.  Returns the list of dL/dA_i."""
    torch = _torch()
    b = len(triplets)
    if b == 0:
        return []
    dt = triplets[0][0].dtype
    ns, ds_, ws = (ctypes.c_int64 * b)(), (ctypes.c_int64 * b)(), (ctypes.c_int32 * b)()
    up, sp, vp, gp, Gp, dp = ((ctypes.c_void_p * b)() for _ in range(6))
    keep, das = [], []
    for i, (u, s, v) in enumerate(triplets):
        u, s, v = u.contiguous(), s.contiguous(), v.contiguous()
        if u.dtype != dt:
            raise ValueError("every triplet must have the same dtype")
        n, w = u.shape
        d = v.shape[0]
        ns[i], ds_[i], ws[i] = n, d, w
        up[i], sp[i], vp[i] = u.data_ptr(), s.data_ptr(), v.data_ptr()
        gs = g_sigmas[i] if g_sigmas is not None else None
        ga = g_aks[i] if g_aks is not None else None
        gs = gs.contiguous().to(dt) if gs is not None else None
        ga = ga.contiguous().to(dt) if ga is not None else None
        if gs is None and ga is None:
            gs = torch.zeros((k,), dtype=dt, device=u.device)
        if gs is not None:
            gp[i] = gs.data_ptr()
        if ga is not None:
            Gp[i] = ga.data_ptr()
        da = torch.empty((n, d), dtype=dt, device=u.device)
        dp[i] = da.data_ptr()
        keep += [u, s, v, gs, ga]
        das.append(da)
    ctx = context(triplets[0][0].device)
    statuses = (ctypes.c_int32 * b)()
    B.check(ctx.lib.bks_backward_batched(ctx.ptr, _dtype_code(dt), b, ctypes.cast(ns, ctypes.c_void_p),
                                         ctypes.cast(ds_, ctypes.c_void_p), int(k), ctypes.cast(ws, ctypes.c_void_p),
                                         ctypes.cast(up, ctypes.c_void_p), ctypes.cast(sp, ctypes.c_void_p),
                                         ctypes.cast(vp, ctypes.c_void_p), ctypes.cast(gp, ctypes.c_void_p),
                                         ctypes.cast(Gp, ctypes.c_void_p), ctypes.cast(dp, ctypes.c_void_p),
                                         float(gap_tau), ctypes.cast(statuses, ctypes.c_void_p)),
            ctx.ptr, "bks_backward_batched")
    return das


# ---------------------------------------------------------------------- batches
def block_krylov_batched(mats, k, q, seeds=None, pis=None, want_v=False, precision="auto", stats=False, **kw):
    """Algorithm 2 on a list of independent matrices (dense CUDA tensors or CsrMatrix) in
    one call (bks_block_krylov_batched).  Returns a list of (Z_i, sigma_i[, V_i]) and,
    with stats, the summed bks_stats and the per-matrix statuses."""
    torch = _torch()
    b = len(mats)
    if b == 0:
        return []
    arr = (BksMatrix * b)()
    outs, zp, sp, vp, pp = [], (ctypes.c_void_p * b)(), (ctypes.c_void_p * b)(), (ctypes.c_void_p * b)(), \
        (ctypes.c_void_p * b)()
    dev = None
    for i, a in enumerate(mats):
        m, dv, odt = _as_bks(a, precision)
        dev = dv if dev is None else dev
        arr[i] = m
        z = torch.empty((m.n, k), dtype=odt, device=dv)
        s = torch.empty((k,), dtype=odt, device=dv)
        v = torch.empty((m.d, k), dtype=odt, device=dv) if want_v else None
        zp[i], sp[i] = z.data_ptr(), s.data_ptr()
        if v is not None:
            vp[i] = v.data_ptr()
        if pis is not None and pis[i] is not None:
            p = pis[i]
            pc = kw.get("block_p") or k
            if p.shape != (m.d, pc) or p.dtype != odt or not p.is_contiguous():
                raise ValueError(f"pis[{i}] must be a contiguous {m.d}x{pc} {odt} tensor")
            pp[i] = p.data_ptr()
        outs.append((z, s, v) if want_v else (z, s))
    ctx = context(dev)
    seeds_arr = (ctypes.c_uint64 * b)(*[int(x) & (2**64 - 1) for x in (seeds if seeds is not None else range(b))])
    statuses = (ctypes.c_int32 * b)()
    opts = _opts(precision=precision, **kw)
    st = BksStats()
    status = ctx.lib.bks_block_krylov_batched(ctx.ptr, b, arr, int(k), int(q), ctypes.cast(seeds_arr, ctypes.c_void_p),
                                              ctypes.cast(pp, ctypes.c_void_p) if pis is not None else None,
                                              ctypes.cast(zp, ctypes.c_void_p), ctypes.cast(sp, ctypes.c_void_p),
                                              ctypes.cast(vp, ctypes.c_void_p) if want_v else None,
                                              ctypes.byref(opts), ctypes.byref(st),
                                              ctypes.cast(statuses, ctypes.c_void_p))
    B.check(status, ctx.ptr, "bks_block_krylov_batched")
    if stats:
        return outs, st.as_dict(), list(statuses)
    return outs
