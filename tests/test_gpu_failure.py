"""Failure paths on the GPU, without a GPU fault.

* A bounded device wait that runs out (bks_selftest_wait: an mbarrier phase and a grid
  barrier that nothing completes) returns BKS_ERR_TIMEOUT after about its 1 s limit, and
  the context solves correctly afterwards.
* A caller workspace smaller than the solve needs returns BKS_ERR_NOMEM before any launch;
  handing the workspace back to the library recovers.
* A block with no independent part left (all zeros) cannot be orthonormalised:
  BKS_ERR_BREAKDOWN, and the context stays usable.
The non-finite path (BKS_ERR_NONFINITE) is covered in test_gpu_dense.py."""
import ctypes
import time

import numpy as np
import pytest

import synth
from oracle import krylov

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def solve_ok():
    """A small solve on the same context, checked against the oracle."""
    a, _, _, _ = synth.dense_planted_small()
    pi = synth.gaussian_pi(1, 300, 10, dtype=np.float64)
    z, s = bk.block_krylov(dev(a), 10, 4, pi=dev(pi))
    ref = krylov.block_krylov(a, 10, 4, pi)
    assert np.max(np.abs(s.cpu().numpy() - ref.sigma) / ref.sigma) < 1e-10


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_context_stays_usable(which):
    ctx = bk.context(torch.device("cuda", 0))
    t0 = time.monotonic()
    st = ctx.lib.bks_selftest_wait(ctx.ptr, which)
    elapsed = time.monotonic() - t0
    assert st == 7, st                      # BKS_ERR_TIMEOUT
    assert 0.9 < elapsed < 30.0, elapsed    # the 1 s limit, not a hang
    assert b"gave up" in ctx.lib.bks_last_error(ctx.ptr)
    assert ctx.lib.bks_selftest_wait(ctx.ptr, 2) == 1   # unknown wait: BKS_ERR_INVALID_ARG
    solve_ok()


def test_caller_workspace_too_small_is_nomem():
    ctx = bk.context(torch.device("cuda", 0))
    small = torch.empty(4096, dtype=torch.uint8, device="cuda")
    ctx.set_workspace(small)
    try:
        with pytest.raises(bk.BksError) as e:
            solve_ok()
        assert e.value.status == 3   # BKS_ERR_NOMEM
        assert "workspace too small" in str(e.value)
    finally:
        ctx.set_workspace(None)
    solve_ok()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_zero_block_is_breakdown(dtype):
    w = torch.zeros((1000, 8), dtype=dtype, device="cuda")
    with pytest.raises(bk.BksError) as e:
        bk.orthonormalize(w)
    assert e.value.status == 5   # BKS_ERR_BREAKDOWN
    q = bk.orthonormalize(torch.randn((1000, 8), dtype=dtype, device="cuda"))
    assert float((q.T @ q - torch.eye(8, dtype=dtype, device="cuda")).abs().max()) < 1e-5
    solve_ok()
