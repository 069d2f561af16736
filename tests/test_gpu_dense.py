"""GPU parity of the dense path against the FP64 oracle, through the C-ABI.

Tolerances (from the arithmetic):
* products: |Y - Y_ref| <= 4 sqrt(K) eps (|A||X|) elementwise, eps of the path's
  precision (FP32 products accumulate K terms in FP32 inside a tile, FP64 across
  split-K partials);
* Ritz values: relative 1e-5 on the FP32 path, 1e-10 on the FP64 path;
* error ratios (eqs. 1-3): within 1e-3 of the oracle's;
* orthonormality: |Q^T Q - I| <= 50 sqrt(n) eps.
"""
import numpy as np
import pytest

import synth
from oracle import krylov, metrics, rng as orng

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")

EPS = {np.float32: 2.0 ** -24, np.float64: 2.0 ** -53}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def align_signs(z, zref):
    s = np.sign(np.sum(z * zref, axis=0))
    s[s == 0] = 1
    return z * s


# ------------------------------------------------------------------ products (a1-a3)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,d,c", [(1000, 300, 7), (517, 1029, 50), (2053, 4099, 64), (33, 17, 1)])
@pytest.mark.parametrize("trans", [False, True])
def test_products_match_fp64(dtype, n, d, c, trans):
    rng = np.random.default_rng(n + d + c)
    a = rng.standard_normal((n, d)).astype(dtype)
    x = rng.standard_normal((n if trans else d, c)).astype(dtype)
    y = host(bk.matmul(dev(a), dev(x), trans=trans))
    a64, x64 = a.astype(np.float64), x.astype(np.float64)
    ref = (a64.T if trans else a64) @ x64
    bound = (np.abs(a64.T if trans else a64) @ np.abs(x64)) * 4 * np.sqrt(x.shape[0]) * EPS[dtype]
    assert y.shape == ref.shape
    assert np.all(np.abs(y - ref) <= bound + 1e-300)


@pytest.mark.parametrize("n,d,c", [(1000, 308, 7), (4093, 1028, 50), (257, 96, 33),
                                   (3001, 2052, 64), (5000, 1000, 100), (1000, 500, 130)])
@pytest.mark.parametrize("trans", [False, True])
def test_tensor_core_products(n, d, c, trans):
    """Shapes whose rows meet the TMA alignment rules take the tcgen05 3xTF32 path; ragged
    tails in both the tiled and the contraction dimension, and more than 128 columns."""
    rng = np.random.default_rng(n + 3 * d + c)
    a = rng.standard_normal((n, d)).astype(np.float32)
    x = rng.standard_normal((n if trans else d, c)).astype(np.float32)
    ad, xd = dev(a), dev(x)
    y = host(bk.matmul(ad, xd, trans=trans))
    y2 = host(bk.matmul(ad, xd, trans=trans))
    ys = host(bk.matmul(ad, xd, trans=trans, simt=True))
    a64, x64 = a.astype(np.float64), x.astype(np.float64)
    ref = (a64.T if trans else a64) @ x64
    bound = (np.abs(a64.T if trans else a64) @ np.abs(x64)) * 4 * np.sqrt(x.shape[0]) * EPS[np.float32]
    assert np.array_equal(y, y2)                       # deterministic
    assert np.all(np.abs(y - ref) <= bound)
    assert np.all(np.abs(ys - ref) <= bound)


@pytest.mark.parametrize("trans", [False, True])
def test_tensor_core_products_unbiased(trans):
    """All-positive data makes every partial sum grow coherently, so an accumulator that
    rounds toward zero shows up as a one-sided relative error of order (steps x 2^-24).
    Round-to-nearest accumulation stays within ~sqrt(K) eps of the exact sum."""
    rng = np.random.default_rng(11)
    n, d, c = 20000, 8000, 50
    a = rng.random((n, d), dtype=np.float32)
    x = rng.random((n if trans else d, c), dtype=np.float32)
    y = host(bk.matmul(dev(a), dev(x), trans=trans)).astype(np.float64)
    ref = (a.astype(np.float64).T if trans else a.astype(np.float64)) @ x.astype(np.float64)
    rel = (y - ref) / ref
    kdim = x.shape[0]
    assert np.max(np.abs(rel)) <= 4 * np.sqrt(kdim) * EPS[np.float32]
    assert abs(np.mean(rel)) <= 0.5 * np.sqrt(kdim) * EPS[np.float32]   # no systematic drift


def test_products_full_size_20000x8000():
    a, _ = synth.dense_planted_noisy()
    rng = np.random.default_rng(5)
    x = rng.standard_normal((8000, 50)).astype(np.float32)
    qx = rng.standard_normal((20000, 50)).astype(np.float32)
    ad = dev(a)
    y = host(bk.matmul(ad, dev(x)))
    b = host(bk.matmul(ad, dev(qx), trans=True))
    a64 = a.astype(np.float64)
    for got, ref, bnd in ((y, a64 @ x, np.abs(a64) @ np.abs(x.astype(np.float64))),
                          (b, a64.T @ qx, np.abs(a64.T) @ np.abs(qx.astype(np.float64)))):
        assert np.all(np.abs(got - ref) <= 4 * np.sqrt(20000) * EPS[np.float32] * bnd)


# --------------------------------------------------------------- orthonormalisation (a4)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n,m,c", [(3001, 0, 9), (3001, 40, 9), (20000, 400, 50), (128, 64, 32)])
def test_orthonormalize(dtype, n, m, c):
    rng = np.random.default_rng(m + c)
    qb = np.linalg.qr(rng.standard_normal((n, m)))[0] if m else None
    w = rng.standard_normal((n, c))
    if m:
        w = w + qb @ rng.standard_normal((m, c)) * 10   # large component inside span(Qb)
    q = host(bk.orthonormalize(dev(w.astype(dtype)), dev(qb.astype(dtype)) if m else None))
    q64 = q.astype(np.float64)
    tol = 50 * np.sqrt(n) * EPS[dtype]
    assert np.max(np.abs(q64.T @ q64 - np.eye(c))) < tol
    resid = w - (qb @ (qb.T @ w) if m else 0)
    if m:
        assert np.max(np.abs(qb.T @ q64)) < tol
    # span(Q) = span of the projected W
    proj = resid - q64 @ (q64.T @ resid)
    assert np.linalg.norm(proj) / np.linalg.norm(resid) < 1e3 * EPS[dtype] * np.sqrt(n)


# ------------------------------------------------------------------ eigen-solve (a6)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("w", [1, 10, 70, 80, 220, 450])
def test_sym_eig(dtype, w):
    rng = np.random.default_rng(w)
    b = rng.standard_normal((w + 30, w)) * np.exp(-np.arange(w) / 40.0)
    m = b.T @ b
    lam, u = bk.sym_eig(dev(m.astype(dtype)))
    lam, u = host(lam).astype(np.float64), host(u).astype(np.float64)
    ref = np.sort(np.linalg.eigvalsh(m))[::-1]
    eps = EPS[dtype]
    assert np.all(np.diff(lam) <= 0)
    assert np.max(np.abs(lam - ref)) <= 100 * np.sqrt(w) * eps * ref[0]
    assert np.max(np.abs(u.T @ u - np.eye(w))) <= 100 * np.sqrt(w) * eps
    assert np.max(np.abs(m @ u - u * lam)) <= 100 * np.sqrt(w) * eps * ref[0]


# ------------------------------------------------------------------ start block (a0)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_device_generator_matches_oracle(dtype):
    """The device generator (CUDA log/sincos in FP64) against the oracle's (glibc):
    FP32 output agrees bit for bit except where the two libms' last-bit differences
    straddle an FP32 rounding boundary; FP64 output agrees to a few ulp."""
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    got = host(bk.gen_pi(77, 8000, 50, dtype=tdt, device="cuda")).astype(np.float64)
    ref = np.empty(8000 * 50)
    for p in range(8000 * 25):
        ref[2 * p], ref[2 * p + 1] = orng.gaussian_pair(77, p)
    ref = ref.reshape(8000, 50)
    if dtype == np.float32:
        ref = ref.astype(np.float32).astype(np.float64)
        assert np.mean(got == ref) > 0.9999
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-30)) <= 2 * EPS[dtype]
    else:
        assert np.max(np.abs(got - ref)) <= 1e-14


# --------------------------------------------------------------- end-to-end (a0-a9)
def _check_solve(a, k, q, method, pi, sig_tol, sigma_true=None):
    fn = bk.block_krylov if method == "bki" else bk.simul_iter
    ofn = krylov.block_krylov if method == "bki" else krylov.simul_iter
    z, s, v = fn(dev(a), k, q, pi=dev(pi), want_v=True)
    z, s, v = host(z).astype(np.float64), host(s).astype(np.float64), host(v).astype(np.float64)
    ref = ofn(a, k, q, pi)
    rel = np.abs(s - ref.sigma) / ref.sigma
    assert np.max(rel) <= sig_tol, (np.max(rel), np.argmax(rel))
    n = a.shape[0]
    eps = EPS[a.dtype.type]
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 100 * np.sqrt(n) * eps + 1e-12
    # V = A^T Z diag(1/sigma)
    a64 = a.astype(np.float64)
    assert np.max(np.abs(v - (a64.T @ z) / s)) < 1e3 * np.sqrt(n) * eps * np.max(np.abs(v))
    r_gpu = metrics.ratios(a64, z, k, sigma=sigma_true)
    r_ora = metrics.ratios(a64, ref.Z, k, sigma=sigma_true)
    for key in r_gpu:
        assert abs(r_gpu[key] - r_ora[key]) <= 1e-3, (key, r_gpu[key], r_ora[key])
    return z, s, ref


@pytest.mark.parametrize("method", ["bki", "si"])
def test_planted_500x300_fp64(method):
    a, sig, _, _ = synth.dense_planted_small()
    pi = synth.gaussian_pi(1, 300, 10, dtype=np.float64)
    z, s, ref = _check_solve(a, 10, 6, method, pi, 1e-10, sigma_true=sig)
    # Ritz vectors agree where the Ritz values are separated
    za = align_signs(z, ref.Z)
    assert np.max(np.abs(za[:, :5] - ref.Z[:, :5])) < 1e-8


@pytest.mark.parametrize("method", ["bki", "si"])
def test_planted_500x300_fp32(method):
    a, sig, _, _ = synth.dense_planted_small()
    a32 = a.astype(np.float32)
    pi = synth.gaussian_pi(1, 300, 10)
    _check_solve(a32, 10, 6, method, pi, 1e-5)


@pytest.mark.parametrize("method", ["bki", "si"])
def test_noisy_scaled_fp32(method):
    a, _ = synth.dense_planted_noisy(n=2000, d=800, rank=200, seed=1002)
    pi = synth.gaussian_pi(2, 800, 50)
    _check_solve(a, 50, 8, method, pi, 1e-5)


@pytest.mark.parametrize("n,d,k,q", [(1003, 517, 7, 3), (5, 3, 1, 0), (64, 48, 16, 2),
                                     (300, 1000, 1, 5), (700, 129, 32, 1)])
def test_ragged_and_small_shapes(n, d, k, q):
    rng = np.random.default_rng(n * d)
    s = np.exp(-np.arange(min(n, d)) / 5.0)
    a, _, _ = synth.planted(n, d, s, n + d)
    pi = rng.standard_normal((d, k))
    for method in ("bki", "si"):
        _check_solve(a, k, q, method, pi, 1e-10)


def test_q_capped_returns_warning_and_exact_values():
    sig = 1.0 / np.arange(1, 49)
    a, _, _ = synth.planted(64, 48, sig, 5)
    z, s, st = bk.block_krylov(dev(a), 16, 4, pi=dev(synth.gaussian_pi(2, 48, 16, np.float64)), stats=True)
    assert st["q_eff"] == 2 and st["width"] == 48
    assert np.allclose(host(s), sig[:16], rtol=1e-10)


def test_seed_path_matches_oracle_start_block():
    a, sig, _, _ = synth.dense_planted_small()
    z, s = bk.block_krylov(dev(a), 10, 4, seed=31)
    ref = krylov.block_krylov(a, 10, 4, orng.start_block(31, 300, 10))
    assert np.max(np.abs(host(s) - ref.sigma) / ref.sigma) < 1e-6


def test_q0_is_sketch_and_solve_on_gpu():
    a, _ = synth.dense_planted_noisy(n=1500, d=600, rank=100, seed=7)
    pi = synth.gaussian_pi(3, 600, 20)
    zb, sb = bk.block_krylov(dev(a), 20, 0, pi=dev(pi))
    zs, ss = bk.simul_iter(dev(a), 20, 0, pi=dev(pi))
    ref = krylov.block_krylov(a, 20, 0, pi)
    assert np.max(np.abs(host(sb) - ref.sigma) / ref.sigma) < 1e-5
    assert np.max(np.abs(host(ss) - ref.sigma) / ref.sigma) < 1e-5


def test_basis_only_returns_orthonormal_basis():
    a, _ = synth.dense_planted_noisy(n=1500, d=600, rank=100, seed=8)
    pi = synth.gaussian_pi(3, 600, 20)
    z, s = bk.block_krylov(dev(a), 20, 3, pi=dev(pi), basis_only=True)
    z = host(z).astype(np.float64)
    assert np.max(np.abs(z.T @ z - np.eye(20))) < 1e-4
    ref = krylov.block_krylov(a, 20, 3, pi)
    # the basis is Q_0, the orthonormalised A Pi
    q0 = ref.Q[:, :20]
    assert metrics.subspace_distance(z, q0) < 1e-4


def test_invalid_arguments_on_gpu():
    a = dev(np.ones((10, 5), np.float32))
    with pytest.raises(bk.BksError) as e:
        bk.block_krylov(a, 6, 1)
    assert e.value.status == 1
    with pytest.raises(bk.BksError):
        bk.block_krylov(a, 0, 1)
    with pytest.raises(bk.BksError):
        bk.block_krylov(a, 2, -1)


def test_nonfinite_input_reported():
    a = np.random.default_rng(0).standard_normal((200, 100)).astype(np.float32)
    a[17, 3] = np.nan
    with pytest.raises(bk.BksError) as e:
        bk.block_krylov(dev(a), 5, 2)
    assert e.value.status == 4   # BKS_ERR_NONFINITE: the NaN reaches the first Gram matrix
    # the context stays usable
    a[17, 3] = 1.0
    z, s = bk.block_krylov(dev(a), 5, 2)
    assert bool(torch.isfinite(s).all())


# ------------------------------------------------------------- full size 20000 x 8000
# The full-size 20000 x 8000 parity test lives in test_gpu_fullsize.py.
