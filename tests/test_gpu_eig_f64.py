"""The FP64 eigen-solve of M on the FP32 and BF16 paths (opts.eig_f64): M is formed as
usual, its eigen-problem solved by the one-sided Jacobi in FP64, the eigenvectors rounded
to FP32.  Parity against the FP64 oracle at the FP32 bar (Ritz values 1e-5 relative, error
ratios within 1e-3, |Z^T Z - I| <= 1e-5) at widths 450 and 160 (BF16, refined)."""
import numpy as np
import pytest

import synth
from oracle import krylov, metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_fp32_width_450():
    a, _ = synth.dense_planted_noisy(n=2000, d=800, rank=200, seed=1002)
    k, q = 50, 8
    pi = synth.gaussian_pi(2, 800, k)
    z, s, st = bk.block_krylov(dev(a), k, q, pi=dev(pi), eig_f64=True, stats=True)
    assert st["eig_path"] == 2 and st["width"] == 450
    z, s = z.double().cpu().numpy(), s.double().cpu().numpy()
    a64 = a.astype(np.float64)
    ref = krylov.block_krylov(a64, k, q, pi.astype(np.float64))
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= 1e-5
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 1e-5
    sig = metrics.true_singular_values(a64)
    r_gpu, r_ora = metrics.ratios(a64, z, k, sigma=sig), metrics.ratios(a64, ref.Z, k, sigma=sig)
    for key in r_gpu:
        assert abs(r_gpu[key] - r_ora[key]) <= 1e-3, key


def test_bf16_refined_width_160():
    a = synth.dense_bf16_planted_torch(m=4096, d=2048, seed=4137, device="cuda")
    a64 = a.float().cpu().numpy().astype(np.float64)
    k, q = 32, 4
    pi = synth.gaussian_pi(4, 2048, k)
    ref = krylov.block_krylov(a64, k, q, pi)
    z, s = bk.block_krylov(a, k, q, pi=dev(pi), precision="bf16", eig_f64=True)
    s = s.double().cpu().numpy()
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= 1e-5
    z = z.double().cpu().numpy()
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 1e-5


def test_ignored_on_the_fp64_path():
    a, _, _, _ = synth.dense_planted_small()
    z, s, st = bk.block_krylov(dev(a), 10, 4, eig_f64=True, stats=True)
    assert st["eig_path"] != 2
