"""GPU parity of the eigen-solve of M = B^T B (step 6 of Algorithms 1 and 2): the
Householder tridiagonal top-k solver (the default when only Ubar_k is returned and
w > k) against the one-sided Jacobi and the FP64 oracle, on spectra chosen to stress it:
fast decay, exactly equal and tightly clustered singular values, a rank below the Krylov
width, and the widest width its kernels take.

Tolerances: Ritz values relative 1e-10 (FP64) / 1e-5 (FP32), as for the Jacobi path;
orthonormality 100 sqrt(n) eps; subspaces of separated groups of singular values within
1e-8 (FP64) / 1e-3 (FP32) of the oracle's."""
import numpy as np
import pytest

import synth
from oracle import krylov, metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")

EPS = {np.float32: 2.0 ** -24, np.float64: 2.0 ** -53}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def solve(a, k, q, pi, **kw):
    z, s, v, st = bk.block_krylov(dev(a), k, q, pi=dev(pi), want_v=True, stats=True, **kw)
    return host(z), host(s), host(v), st


def spectrum(kind, r):
    if kind == "decay":
        return np.exp(-np.arange(r) / 8.0)
    if kind == "equal":   # groups of exactly equal singular values
        return np.concatenate([np.full(4, 3.0), np.full(3, 2.0), np.exp(-np.arange(r - 7) / 6.0)])
    if kind == "cluster":  # relative gaps of 1e-7 inside the leading group
        return np.concatenate([1.0 + 1e-7 * np.arange(5)[::-1], 0.5 * np.exp(-np.arange(r - 5) / 6.0)])
    raise ValueError(kind)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("kind", ["decay", "equal", "cluster"])
def test_tridiagonal_matches_oracle_and_jacobi(dtype, kind):
    n, d, k, q = 600, 400, 12, 4
    sig = spectrum(kind, 400)
    a, _, _ = synth.planted(n, d, sig, 77)
    a = a.astype(dtype)
    pi = synth.gaussian_pi(8, d, k).astype(dtype)
    z, s, v, st = solve(a, k, q, pi)
    zj, sj, vj, stj = solve(a, k, q, pi, eig_mode="jacobi")
    assert st["eig_path"] == 1 and stj["eig_path"] == 0 and st["jacobi_sweeps"] == 0
    ref = krylov.block_krylov(a.astype(np.float64), k, q, pi.astype(np.float64))
    tol = 1e-10 if dtype == np.float64 else 1e-5
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= tol
    assert np.max(np.abs(s - sj) / sj) <= tol
    eps = EPS[dtype]
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 100 * np.sqrt(n) * eps + 1e-12
    # V = A^T Z diag(1/sigma)
    assert np.max(np.abs(v - (a.astype(np.float64).T @ z) / s)) < 1e3 * np.sqrt(n) * eps * np.max(np.abs(v))
    # groups separated from the rest: same subspace as the oracle's
    groups = {"decay": [(0, 1), (0, 6), (0, 12)], "equal": [(0, 4), (4, 7), (0, 12)],
              "cluster": [(0, 5), (0, 12)]}[kind]
    stol = 1e-8 if dtype == np.float64 else 1e-3
    for g0, g1 in groups:
        assert metrics.subspace_distance(z[:, g0:g1], ref.Z[:, g0:g1]) < stol, (g0, g1)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_rank_below_krylov_width(dtype):
    """rank(A) = 20 < w: M has w - 20 eigenvalues at rounding level, one large cluster for
    the inverse iteration; with k = 25 five Ritz vectors lie in the numerical null space,
    where the Krylov basis itself is only as orthonormal as the shifted CholeskyQR2 of a
    rank-deficient block makes it, so orthonormality is checked on the leading 20."""
    n, d, r = 500, 300, 20
    rng = np.random.default_rng(5)
    u = np.linalg.qr(rng.standard_normal((n, r)))[0]
    w_ = np.linalg.qr(rng.standard_normal((d, r)))[0]
    a = ((u * np.linspace(2.0, 1.0, r)) @ w_.T).astype(dtype)
    for k, q in ((10, 5), (25, 1)):
        pi = synth.gaussian_pi(9, d, k).astype(dtype)
        z, s, v, st = solve(a, k, q, pi)
        assert st["eig_path"] == 1
        eps = EPS[dtype]
        top = min(k, r)
        zt = z[:, :top]
        assert np.max(np.abs(zt.T @ zt - np.eye(top))) < 100 * np.sqrt(n) * eps + 1e-12
        ref = np.linspace(2.0, 1.0, r)[:top]
        assert np.max(np.abs(s[:top] - ref) / ref) < (1e-10 if dtype == np.float64 else 1e-5)
        if k > r:
            assert np.max(s[r:]) < 1e-3 * s[0]


def test_widest_fp32_width():
    """w = 700 (k = 100, q = 6): the tridiagonal reduction runs on a 16-CTA cluster."""
    n, d, k, q = 3000, 1500, 100, 6
    sig = 1.0 / np.sqrt(np.arange(1, 1501))
    a, _, _ = synth.planted(n, d, sig, 13)
    a = a.astype(np.float32)
    pi = synth.gaussian_pi(10, d, k)
    z, s, v, st = solve(a, k, q, pi)
    assert st["eig_path"] == 1 and st["width"] == 700
    ref = krylov.block_krylov(a.astype(np.float64), k, q, pi.astype(np.float64))
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= 1e-5
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 100 * np.sqrt(n) * EPS[np.float32]


def test_fp64_width_with_two_ring_slots():
    """w = 500 (k = 50, q = 9) in FP64: the tridiagonal reduction's cluster holds 32
    columns per CTA, and the back-transformation's ring of reflector blocks has only two
    slots at this width (each bulk-copy slot is refilled every other block)."""
    n, d, k, q = 1200, 700, 50, 9
    sig = np.exp(-np.arange(700) / 60.0)
    a, _, _ = synth.planted(n, d, sig, 21)
    pi = synth.gaussian_pi(12, d, k, dtype=np.float64)
    z, s, v, st = solve(a, k, q, pi)
    assert st["eig_path"] == 1 and st["width"] == 500
    ref = krylov.block_krylov(a, k, q, pi)
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= 1e-10
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 100 * np.sqrt(n) * EPS[np.float64]
    # the leading group is well separated: the same subspace as the oracle's
    assert metrics.subspace_distance(z[:, :10], ref.Z[:, :10]) < 1e-8


def test_jacobi_kept_where_all_vectors_or_w_equals_k():
    a, _ = synth.dense_planted_noisy(n=1500, d=600, rank=100, seed=9)
    pi = synth.gaussian_pi(3, 600, 20)
    _, _, st = bk.simul_iter(dev(a), 20, 3, pi=dev(pi), stats=True)
    assert st["eig_path"] == 0
    _, _, st = bk.block_krylov(dev(a), 20, 3, pi=dev(pi), stats=True, rr_mode="qr")
    assert st["eig_path"] == 0
    u, s, v = bk.ritz_triplets(dev(a), 20, 3, pi=dev(pi))
    z, s2 = bk.block_krylov(dev(a), 20, 3, pi=dev(pi))
    assert np.max(np.abs(host(s)[:20] - host(s2)) / host(s2)) < 1e-5
