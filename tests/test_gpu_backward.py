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


def loss_of(sk, ak, t):
    return sk.sum() + ((ak - t) ** 2).sum()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_recompute_mode_is_bit_identical(dtype):
    """recompute=True keeps only A and Pi between forward and backward and solves again in
    the backward; the solve is deterministic, so the gradient is the same to the bit."""
    a, t = case(300, 200, 21)
    k, q = 16, 4
    npdt = np.float64 if dtype == torch.float64 else np.float32
    pi = cuda(synth.gaussian_pi(5, 200, k).astype(npdt), dtype)
    grads = []
    for rec in (False, True):
        at = cuda(a, dtype).requires_grad_(True)
        sk, ak = bk.rand_svd(at, k, q, pi=pi, recompute=rec)
        loss_of(sk, ak, cuda(t, dtype)).backward()
        grads.append(at.grad.clone())
    assert torch.equal(grads[0], grads[1])


def test_recompute_mode_keeps_no_triplets():
    n, d, k, q = 2000, 1000, 16, 4
    a = cuda(np.random.default_rng(5).standard_normal((n, d)), torch.float32)
    w = bk.krylov_width(n, d, k, q)
    held = {}
    for rec in (False, True):
        at = a.clone().requires_grad_(True)
        torch.cuda.synchronize()
        base = torch.cuda.memory_allocated()
        sk, ak = bk.rand_svd(at, k, q, seed=3, recompute=rec)
        torch.cuda.synchronize()
        held[rec] = torch.cuda.memory_allocated() - base
        del sk, ak
    assert held[False] - held[True] >= (n + d + 1) * w * 4   # U, sigma and V are not held


@pytest.mark.parametrize("recompute", [False, True])
def test_batched_forward_backward_matches_oracle_and_single(recompute):
    """Uneven shapes whose Krylov width covers min(n, d) (k = 16, q = 4: width 48, 64 or 80
    after the cap), where the gradient is exact: every matrix's gradient matches the FP64
    oracle's loss gradient, and the batched forward + backward equal the single calls (made
    with the batch's SM budget) bit for bit."""
    shapes = [(64, 48), (120, 64), (80, 200), (96, 80), (48, 300), (256, 64)]
    k, q = 16, 4
    mats, targets = [], []
    for i, (n, d) in enumerate(shapes):
        a, t = case(n, d, 700 + i)
        mats.append(a)
        targets.append(t)
    pis = [cuda(synth.gaussian_pi(30 + i, d, k).astype(np.float64), torch.float64)
           for i, (_, d) in enumerate(shapes)]
    ats = [cuda(a, torch.float64).requires_grad_(True) for a in mats]
    outs = bk.rand_svd_batched(ats, k, q, pis=pis, recompute=recompute)
    sum(loss_of(sk, ak, cuda(t, torch.float64)) for (sk, ak), t in zip(outs, targets)).backward()
    for i, (a, t) in enumerate(zip(mats, targets)):
        g_ora = grad.loss_grad(a, k, t)
        assert rel(ats[i].grad.cpu().numpy(), g_ora) < 1e-7, i
        single = cuda(a, torch.float64).requires_grad_(True)
        sk, ak = bk.rand_svd(single, k, q, pi=pis[i], max_sms=bk.batch_budget(ats, k, q))
        loss_of(sk, ak, cuda(t, torch.float64)).backward()
        assert torch.equal(single.grad, ats[i].grad), i
        assert torch.equal(sk, outs[i][0]) and torch.equal(ak, outs[i][1]), i


def test_batched_uneven_workload_equals_single():
    """Twelve FP32 matrices of the batched workload's shape ranges (m in [256, 4096], n in
    [128, 2048]), seeds 0..11: the batched gradients equal the single calls' bit for bit."""
    mats = synth.batched_planted(batch=12, seed=1005)
    k, q = 16, 4
    ts = [synth.loss_target(90 + i, *m.shape).astype(np.float32) for i, m in enumerate(mats)]
    ats = [cuda(a, torch.float32).requires_grad_(True) for a in mats]
    outs = bk.rand_svd_batched(ats, k, q)
    sum(loss_of(sk, ak, cuda(t, torch.float32)) for (sk, ak), t in zip(outs, ts)).backward()
    for i, (a, t) in enumerate(zip(mats, ts)):
        single = cuda(a, torch.float32).requires_grad_(True)
        sk, ak = bk.rand_svd(single, k, q, seed=i, max_sms=bk.batch_budget(ats, k, q))
        loss_of(sk, ak, cuda(t, torch.float32)).backward()
        assert torch.equal(single.grad, ats[i].grad), i


@pytest.mark.parametrize("d", [512, 510])
def test_backward_products_match_the_oracle_formula(d):
    """FP32 backward at 1024 x d, k = 16, q = 4 (width 80, below the rank): the two passes
    over G run on the tensor cores for d = 512 and on the CUDA cores for d = 510 (rows not
    16-byte aligned).  Both match the oracle's formula evaluated in FP64 on the same
    triplets; the FP32 error is amplified by 1 / (lambda_16 - lambda_17) in the c_ij terms."""
    n, k, q = 1024, 16, 4
    a, _ = case(n, d, 77)
    at = cuda(a, torch.float32)
    u, s, v = bk.ritz_triplets(at, k, q, seed=9)
    rng = np.random.default_rng(8)
    gs = rng.standard_normal(k)
    gg = rng.standard_normal((n, d))
    got = bk.backward(u, s, v, k, cuda(gs, torch.float32), cuda(gg, torch.float32)).double().cpu().numpy()
    un, sn, vn = (x.double().cpu().numpy() for x in (u, s, v))
    ref = grad.adjoint_from_triplets(un, sn, vn, k, gs, gg, gap_tau=1e-6)
    assert rel(got, ref) < 1e-3
