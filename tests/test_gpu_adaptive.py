"""GPU parity of Block Krylov Iteration with the iteration count chosen on the fly
(bks_block_krylov_adaptive) against the FP64 oracle's same rule: the GPU stops after the
same number of iterations and then returns what bks_block_krylov returns at that q.

The tolerance handed to both is the geometric mean of two consecutive relative changes
the oracle observes (a factor >= 2 apart), so that FP32 rounding of the changes (~1e-6)
cannot move the stopping iteration."""
import numpy as np
import pytest

import synth
from oracle import krylov

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def pick_tol(deltas, below):
    """Tolerance between the first change under `below` and the one before it."""
    for j in range(1, len(deltas)):
        if deltas[j] < below and deltas[j - 1] >= 2 * deltas[j]:
            return float(np.sqrt(deltas[j - 1] * deltas[j])), j + 1   # stops with q = j + 1
    raise AssertionError(f"no usable change sequence: {deltas}")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_adaptive_stops_where_the_oracle_stops(dtype):
    a, _ = synth.dense_planted_noisy(n=2000, d=800, rank=200, seed=1002)
    a = a.astype(dtype)
    k, q_max = 20, 10
    pi = synth.gaussian_pi(5, 800, k).astype(dtype)
    _, deltas = krylov.block_krylov_adaptive(a.astype(np.float64), k, q_max, 1e-300, pi.astype(np.float64))
    tol, q_stop = pick_tol(deltas, 1e-2)
    ref, _ = krylov.block_krylov_adaptive(a.astype(np.float64), k, q_max, tol, pi.astype(np.float64))
    assert ref.q_eff == q_stop
    z, s, st = bk.block_krylov_adaptive(dev(a), k, q_max, tol, pi=dev(pi), stats=True)
    assert st["q_eff"] == q_stop and st["width"] == k * (q_stop + 1)
    rtol = 1e-10 if dtype == np.float64 else 1e-5
    assert np.max(np.abs(host(s) - ref.sigma) / ref.sigma) <= rtol
    # the answer is bks_block_krylov's at the iteration count chosen
    z1, s1 = bk.block_krylov(dev(a), k, q_stop, pi=dev(pi))
    assert torch.equal(z, z1) and torch.equal(s, s1)


def test_adaptive_centred_csr():
    n, d, k, q_max = 3000, 1500, 10, 12
    row_ptr, col_idx, vals, d = synth.zipf_idf_csr(n=n, d=d, per_row=30, seed=9)
    mu = synth.column_means(row_ptr, col_idx, vals, n, d)
    a = bk.CsrMatrix(dev(row_ptr), dev(col_idx), dev(vals), (n, d), col_mean=dev(mu))
    pi = synth.gaussian_pi(3, d, k)
    op = krylov.centred_csr_op(row_ptr, col_idx, vals, n, d, mu)
    _, deltas = krylov.block_krylov_adaptive(op, k, q_max, 1e-300, pi)
    tol, q_stop = pick_tol(deltas, 3e-3)
    ref, _ = krylov.block_krylov_adaptive(op, k, q_max, tol, pi)
    z, s, st = bk.block_krylov_adaptive(a, k, q_max, tol, pi=dev(pi), stats=True)
    assert st["q_eff"] == ref.q_eff == q_stop
    assert np.max(np.abs(host(s) - ref.sigma) / ref.sigma) <= 1e-5


def test_adaptive_runs_q_max_without_convergence_and_takes_block_p():
    a, _, _, _ = synth.dense_planted_small()
    z, s, st = bk.block_krylov_adaptive(dev(a), 10, 3, 1e-14, seed=4, stats=True)
    assert st["q_eff"] == 3
    z1, s1 = bk.block_krylov(dev(a), 10, 3, seed=4)
    assert torch.equal(s, s1)
    z, s, st = bk.block_krylov_adaptive(dev(a), 10, 6, 1e-3, seed=4, stats=True, block_p=16)
    assert 1 <= st["q_eff"] <= 6 and st["width"] == 16 * (st["q_eff"] + 1)


def test_adaptive_rejects_bad_tolerance():
    a = dev(np.random.default_rng(0).standard_normal((60, 40)).astype(np.float32))
    for tol in (0.0, -1.0, 1.5):
        with pytest.raises(bk.BksError):
            bk.block_krylov_adaptive(a, 5, 3, tol)
