"""GPU parity of the differentiation path: Ritz triplets, the rank-k reconstruction and
bks_backward, against the FP64 oracle adjoint (oracle.grad) and central differences, on
the 64 x 48 case of the batched workload (sigma_i = 1/i plus 1e-3 N(0,1), k = 16, q = 4,
so q is capped to 2 and the Krylov width 48 covers range(A): the formula is exact).

Tolerances: FP64 path 1e-7 relative (the oracle pin's own level), FP32 path 1e-4."""
import numpy as np
import pytest

import synth
from oracle import grad, krylov

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")


def case(n=64, d=48, seed=1005):
    rg = np.random.default_rng(seed)
    sig = 1.0 / np.arange(1, min(n, d) + 1)
    a, _, _ = synth.planted(n, d, sig, seed)
    a = a + 1e-3 * rg.standard_normal((n, d))
    t = synth.loss_target(77, n, d)
    return a, t


def cuda(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-7), (torch.float32, 1e-4)])
def test_loss_gradient_matches_oracle_and_differences(dtype, tol):
    a, t = case()
    k, q = 16, 4
    pi = synth.gaussian_pi(5, 48, k).astype(np.float64 if dtype == torch.float64 else np.float32)
    at = cuda(a, dtype).requires_grad_(True)
    sk, ak = bk.rand_svd(at, k, q, pi=cuda(pi, dtype))
    loss = sk.sum() + ((ak - cuda(t, dtype)) ** 2).sum()
    loss.backward()
    g_gpu = at.grad.double().cpu().numpy()
    g_ora = grad.loss_grad(a, k, t)
    assert rel(g_gpu, g_ora) < tol
    if dtype == torch.float64:
        g_fd = grad.central_difference(a, k, t)
        assert rel(g_gpu, g_fd) < 1e-6


def test_backward_terms_separately():
    a, t = case()
    k, q = 16, 4
    at = cuda(a, torch.float64)
    u, s, v = bk.ritz_triplets(at, k, q, pi=cuda(synth.gaussian_pi(5, 48, k).astype(np.float64), torch.float64))
    rng = np.random.default_rng(3)
    gs = rng.standard_normal(k)
    gg = rng.standard_normal(a.shape)
    only_s = bk.backward(u, s, v, k, g_sigma=cuda(gs, torch.float64)).cpu().numpy()
    only_g = bk.backward(u, s, v, k, g_ak=cuda(gg, torch.float64)).cpu().numpy()
    both = bk.backward(u, s, v, k, cuda(gs, torch.float64), cuda(gg, torch.float64)).cpu().numpy()
    assert rel(only_s, grad.adjoint(a, k, gs, None)) < 1e-9
    assert rel(only_g, grad.adjoint(a, k, np.zeros(k), gg)) < 1e-8
    assert rel(both, only_s + only_g) < 1e-12
    with pytest.raises(bk.BksError):
        bk.backward(u, s, v, k)


@pytest.mark.parametrize("method", ["bki", "si"])
def test_ritz_triplets_extend_the_solve(method):
    a, _ = case(300, 200, 11)
    k, q = 10, 4
    at = cuda(a, torch.float64)
    pi = cuda(synth.gaussian_pi(6, 200, k).astype(np.float64), torch.float64)
    u, s, v = bk.ritz_triplets(at, k, q, pi=pi, method=method)
    w = bk.krylov_width(300, 200, k, q, method)
    assert u.shape == (300, w) and s.shape == (w,) and v.shape == (200, w)
    fn = bk.block_krylov if method == "bki" else bk.simul_iter
    z, sig, vk = fn(at, k, q, pi=pi, want_v=True)
    un, sn, vn = (x.cpu().numpy() for x in (u, s, v))
    assert np.max(np.abs(sn[:k] - sig.cpu().numpy()) / sig.cpu().numpy()) < 1e-12
    assert np.max(np.abs(un[:, :k] - z.cpu().numpy())) < 1e-10
    assert np.max(np.abs(vn[:, :k] - vk.cpu().numpy())) < 1e-10
    assert np.all(np.diff(sn) <= 0)
    assert np.max(np.abs(un.T @ un - np.eye(w))) < 1e-12
    assert np.max(np.abs(a.T @ un - vn * sn)) < 1e-10 * sn[0]
    ref = (krylov.block_krylov if method == "bki" else krylov.simul_iter)(a, k, q, pi.cpu().numpy())
    assert np.max(np.abs(sn[:k] - ref.sigma) / ref.sigma) < 1e-10


def test_low_rank_reconstruction():
    a, _ = case()
    at = cuda(a, torch.float32)
    u, s, v = bk.ritz_triplets(at, 16, 4)
    ak = bk.low_rank(u, s, v, 16).double().cpu().numpy()
    un, sn, vn = (x.double().cpu().numpy() for x in (u, s, v))
    ref = (un[:, :16] * sn[:16]) @ vn[:, :16].T
    assert np.max(np.abs(ak - ref)) < 1e-6 * np.max(np.abs(ref))
    # A_k = Z Z^T A
    assert np.max(np.abs(ak - un[:, :16] @ (un[:, :16].T @ a))) < 1e-5
