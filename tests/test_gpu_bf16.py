"""GPU parity of the mixed-precision path (dense BF16 A): the kind::f16 tensor-core
products in both of their forms, and the BF16-mode solve with and without the FP32
refinement pass, against the FP64 oracle run on the exact upcast of the BF16 matrix.

Tolerances.  Exact products (three BF16 pieces of X) carry only FP32 accumulation error:
|Y - Y_ref| <= 4 sqrt(K) eps32 (|A| |X|).  BF16-mode products are compared with the
FP64 product of A and X rounded to BF16 (the operands the tensor cores see), to the same
bound.  The solve in "f32" precision on a BF16 A follows the FP32 bar (relative sigma
1e-5).  The BF16 mode rounds the thin operands of the Krylov products to BF16, so its
basis is not the oracle's; the refinement recomputes B = A^T Q FP32-accurately on that
basis.  For Block Krylov the leading Ritz values are converged directions of a wide
space, which a perturbation of the basis moves only at second order: relative sigma 1e-5
with refinement, 3e-4 without (measured 1.3e-4 at width 100).  Simultaneous Iteration's
k-dimensional space is far from converged at q = 4 on the slowly decaying i^-1/2
spectrum, and the BF16 rounding of its iterates moves the Ritz values at first order:
1e-3 in both forms (measured 1.3e-4 and 3.4e-4 with refinement).  Every form keeps the
error ratios within 1e-3 of the oracle's."""
import numpy as np
import pytest

import synth
from oracle import krylov, metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")

EPS32 = 2.0 ** -24


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def rand_bf16(n, d, seed, positive=False):
    g = torch.Generator().manual_seed(seed)
    a = torch.rand((n, d), generator=g) if positive else torch.randn((n, d), generator=g)
    return a.to(torch.bfloat16)


def check_product(a_bf16, x, y, trans, round_x):
    a64 = a_bf16.float().numpy().astype(np.float64)
    m = a64.T if trans else a64
    xr = synth.bf16_round(x) if round_x else x
    ref = m @ xr.astype(np.float64)
    absd = np.abs(m) @ np.abs(xr.astype(np.float64))
    k = m.shape[1]
    bound = 4 * np.sqrt(k) * EPS32 * absd + 1e-30
    err = np.abs(y - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


SHAPES = [(1000, 512), (777, 328), (129, 72), (3000, 1024)]


@pytest.mark.parametrize("n,d", SHAPES)
@pytest.mark.parametrize("c", [1, 20, 100, 130])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("exact", [True, False])
def test_bf16_products(n, d, c, trans, exact):
    a = rand_bf16(n, d, 7 + n + d)
    rng = np.random.default_rng(c)
    x = rng.standard_normal((n if trans else d, c)).astype(np.float32)
    y = host(bk.matmul(a.cuda(), dev(x), trans=trans, exact=exact))
    check_product(a, x, y, trans, round_x=not exact)
    y2 = host(bk.matmul(a.cuda(), dev(x), trans=trans, exact=exact))
    assert np.array_equal(y, y2)   # deterministic


@pytest.mark.parametrize("trans", [False, True])
def test_bf16_products_unaligned_rows_use_cuda_cores(trans):
    """d not a multiple of 8: the TMA rules fail and the CUDA-core kernel runs (FP32-
    accurate in both forms)."""
    n, d, c = 500, 300, 20
    a = rand_bf16(n, d, 3)
    x = np.random.default_rng(4).standard_normal((n if trans else d, c)).astype(np.float32)
    y = host(bk.matmul(a.cuda(), dev(x), trans=trans, exact=True))
    check_product(a, x, y, trans, round_x=False)


@pytest.mark.parametrize("trans", [False, True])
def test_bf16_exact_products_unbiased(trans):
    """All-positive operands over a long contraction: truncating FP32 accumulation would
    show as a one-signed relative error; the windowed register sums keep the mean error
    at rounding level."""
    n, d, c = 16384, 4096, 32
    a = rand_bf16(n, d, 11, positive=True)
    x = np.random.default_rng(5).random((n if trans else d, c)).astype(np.float32)
    y = host(bk.matmul(a.cuda(), dev(x), trans=trans, exact=True))
    a64 = a.float().numpy().astype(np.float64)
    ref = (a64.T if trans else a64) @ x.astype(np.float64)
    rel = (y - ref) / ref
    kdim = x.shape[0]
    assert np.max(np.abs(rel)) <= 4 * np.sqrt(kdim) * EPS32
    assert abs(np.mean(rel)) <= 0.5 * np.sqrt(kdim) * EPS32   # no systematic drift


def _planted(m, d, seed):
    a = synth.dense_bf16_planted_torch(m=m, d=d, seed=seed, device="cuda")
    return a, a.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("method", ["bki", "si"])
@pytest.mark.parametrize("m,d,k,q", [(2048, 1024, 20, 4), (4096, 2048, 32, 4)])
def test_bf16_solve_small_parity(method, m, d, k, q):
    """Width 100 and 160 (Block Krylov): the refinement of B = A^T Q then runs on one and
    on two groups of 128 columns."""
    a, a64 = _planted(m, d, 41 + m)
    pi = synth.gaussian_pi(4, d, k)
    ref = (krylov.block_krylov if method == "bki" else krylov.simul_iter)(a64, k, q, pi)
    sig = metrics.true_singular_values(a64)
    r_ora = metrics.ratios(a64, ref.Z, k, sigma=sig)
    fn = bk.block_krylov if method == "bki" else bk.simul_iter
    bki = method == "bki"
    cases = {"f32": (dict(precision="f32"), 1e-5, 1e-3),
             "bf16_refined": (dict(precision="bf16"), 1e-5 if bki else 1e-3, 1e-3),
             "bf16_plain": (dict(precision="bf16", refine=False), 3e-4 if bki else 1e-3, 1e-3)}
    for name, (kw, s_tol, r_tol) in cases.items():
        z, s = fn(a, k, q, pi=dev(pi), **kw)
        z, s = host(z), host(s)
        rel = np.max(np.abs(s - ref.sigma) / ref.sigma)
        assert rel <= s_tol, (name, rel)
        orth = np.max(np.abs(z.T @ z - np.eye(k)))
        assert orth < 1e-5, (name, orth)
        r = metrics.ratios(a64, z, k, sigma=sig)
        for key in r:
            assert abs(r[key] - r_ora[key]) <= r_tol, (name, key, r[key], r_ora[key])


def test_bf16_mode_rejects_fp32_matrix():
    a = torch.randn(64, 32, device="cuda")
    with pytest.raises(bk.BksError) as err:
        bk.block_krylov(a, 4, 2, precision="bf16")
    assert err.value.status == 8


def test_bf16_stats_count_the_refinement_pass():
    m, d, k, q = 2048, 1024, 20, 4
    a, _ = _planted(m, d, 41)
    _, _, st = bk.block_krylov(a, k, q, seed=3, precision="bf16", stats=True)
    _, _, st0 = bk.block_krylov(a, k, q, seed=3, precision="bf16", refine=False, stats=True)
    w = k * (q + 1)
    assert st["width"] == w
    nd = float(m) * d
    assert st0["product_flops"] == pytest.approx((2 * q + 2) * 2 * k * nd)
    assert st["product_flops"] == pytest.approx((2 * q + 2) * 2 * k * nd + 2 * (w - k) * nd)
