"""The allocation-free eigen-solve entry point against the regular one.

bks_sym_eig_noalloc serves callers that cannot allocate device memory at call time;
it keeps its scratch in a static device array inside the library.  This file runs
last (pytest collects it after the others) so a failure here never hides another
test's result; it passes both on its own in a fresh process and after the rest of
the suite, because the regular entry point is exercised through its own context
while this one uses no context at all."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")
from paper_1504_05477_gb300 import _binding as B  # noqa: E402

EPS = {torch.float32: 2.0 ** -24, torch.float64: 2.0 ** -53}


def _psd(w, seed):
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((w + 30, w)) * np.exp(-np.arange(w) / 40.0)
    return b.T @ b


def _noalloc(m):
    lib = B.load()
    w = m.shape[0]
    lam = torch.empty((w,), dtype=m.dtype, device=m.device)
    u = torch.empty((w, w), dtype=m.dtype, device=m.device)
    stream = torch.cuda.current_stream(m.device).cuda_stream
    code = B.BKS_F64 if m.dtype == torch.float64 else B.BKS_F32
    status = lib.bks_sym_eig_noalloc(ctypes.c_void_p(stream), code, w, ctypes.c_void_p(m.data_ptr()),
                                     m.stride(0), ctypes.c_void_p(lam.data_ptr()),
                                     ctypes.c_void_p(u.data_ptr()), u.stride(0))
    assert status == B.BKS_OK, status
    return lam, u


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_matches_regular_entry_point_twice(dtype):
    # w = 512 is BKS_NOALLOC_EIG_MAX_W: the layout that sizes the static array (FP64) and
    # the widest Jacobi plan; 450 and 70 are the widths of two solves of the benchmarks
    for call, (w, seed) in enumerate([(450, 1), (70, 2), (512, 3), (512, 4)]):
        m = torch.from_numpy(_psd(w, seed)).to(device="cuda", dtype=dtype).contiguous()
        lam_n, u_n = _noalloc(m)
        lam_r, u_r = bk.sym_eig(m)
        lam_n, u_n = lam_n.cpu().double().numpy(), u_n.cpu().double().numpy()
        lam_r, u_r = lam_r.cpu().double().numpy(), u_r.cpu().double().numpy()
        # both entry points launch the same deterministic kernels on the same plan and
        # leading dimensions, only from different scratch memory: the results are the
        # same bits (a wrong offset in the static layout would break this)
        assert np.array_equal(lam_n, lam_r), call
        assert np.array_equal(u_n, u_r), call
        # and the eigen-solve itself is sound: eigenvalues against LAPACK
        ref = np.linalg.eigvalsh(m.cpu().double().numpy())[::-1]
        tol = 100 * np.sqrt(w) * EPS[dtype]
        assert np.max(np.abs(lam_n - ref)) <= tol * ref[0], call


def test_noalloc_rejects_sizes_beyond_the_limit():
    lib = B.load()
    w = 513   # one above BKS_NOALLOC_EIG_MAX_W
    m = torch.zeros((w, w), device="cuda")
    out = torch.zeros((w,), device="cuda")
    u = torch.zeros((w, w), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    status = lib.bks_sym_eig_noalloc(ctypes.c_void_p(stream), B.BKS_F32, w, ctypes.c_void_p(m.data_ptr()),
                                     w, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(u.data_ptr()), w)
    assert status == B.BKS_ERR_INVALID_ARG
