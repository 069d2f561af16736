"""GPU parity of Block Lanczos (Sec. 4; bks_block_lanczos) against the FP64 oracle
(oracle/lanczos.py), through the C-ABI.

The GPU forms only the block-tridiagonal band of T = Q^T A A^T Q (D_j = B_j^T B_j,
R_{j-1} = B_j^T B_{j-1}) and runs the three-term recurrence before the reorthogonalisation
chosen by `reorth`; the oracle does the same in FP64 with Householder QR.  Tolerances as
for Algorithm 2 (tests/test_gpu_dense.py): Ritz values relative 1e-10 (FP64) and 1e-5
(FP32), error ratios within 1e-3 of the oracle's, |Z^T Z - I| <= 100 sqrt(n) eps where Q
stays orthonormal (full reorthogonalisation, and any mode before the Ritz values converge).
Without full reorthogonalisation Q drifts from orthogonality as Ritz values converge; the
top-k values stay accurate while the drift is small (the FP64 oracle shows the same), so
those cases compare the values only, and one FP32 case shows the drift growing into
spurious copies of converged values.
"""
import numpy as np
import pytest

import synth
from oracle import krylov, lanczos, metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")

EPS = {np.float32: 2.0 ** -24, np.float64: 2.0 ** -53}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def align_signs(z, zref):
    s = np.sign(np.sum(z * zref, axis=0))
    s[s == 0] = 1
    return z * s


def run(a, k, q, pi, reorth, **kw):
    z, s, v, st = bk.block_lanczos(dev(a), k, q, pi=dev(pi), reorth=reorth, want_v=True, stats=True, **kw)
    return host(z), host(s), host(v), st


def check_values(s, ref, tol):
    rel = np.max(np.abs(s - ref.sigma) / ref.sigma)
    assert rel <= tol, rel


def check_vectors(a, z, s, v, k, eps):
    n = a.shape[0]
    a64 = a.astype(np.float64)
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 100 * np.sqrt(n) * eps + 1e-12
    assert np.max(np.abs(v - (a64.T @ z) / s)) < 1e3 * np.sqrt(n) * eps * np.max(np.abs(v))


# ------------------------------------------------------------------ FP64
@pytest.mark.parametrize("reorth,q", [("full", 3), ("full", 6), ("local", 3), ("none", 2)])
def test_fp64_planted_500x300(reorth, q):
    a, sig, _, _ = synth.dense_planted_small()
    k = 10
    pi = synth.gaussian_pi(1, 300, k, dtype=np.float64)
    z, s, v, st = run(a, k, q, pi, reorth)
    ref = lanczos.block_lanczos(a, k, q, pi, reorth=reorth)
    assert st["width"] == k * (q + 1) and st["q_eff"] == q
    check_values(s, ref, 1e-10)
    check_vectors(a, z, s, v, k, EPS[np.float64])
    za = align_signs(z, ref.Z)
    assert np.max(np.abs(za[:, :5] - ref.Z[:, :5])) < 1e-8   # separated Ritz values
    r_gpu = metrics.ratios(a, z, k, sigma=sig)
    r_ora = metrics.ratios(a, ref.Z, k, sigma=sig)
    for key in r_gpu:
        assert abs(r_gpu[key] - r_ora[key]) <= 1e-3, key


def test_fp64_local_after_orthogonality_is_lost():
    """q = 6 on the 500 x 300 matrix: the FP64 oracle's local basis drifts by ~1e-2 from
    orthogonality, yet its top-k Ritz values equal those of the full method."""
    a, _, _, _ = synth.dense_planted_small()
    k, q = 10, 6
    pi = synth.gaussian_pi(1, 300, k, dtype=np.float64)
    _, s, _, _ = run(a, k, q, pi, "local")
    full = lanczos.block_lanczos(a, k, q, pi, reorth="full")
    check_values(s, full, 1e-9)


@pytest.mark.parametrize("n,d,k,q", [(1003, 517, 7, 3), (300, 1000, 1, 5), (700, 129, 32, 1), (5, 3, 1, 0)])
def test_fp64_ragged_shapes(n, d, k, q):
    rng = np.random.default_rng(n * d + 1)
    s_true = np.exp(-np.arange(min(n, d)) / 5.0)
    a, _, _ = synth.planted(n, d, s_true, n + d)
    pi = rng.standard_normal((d, k))
    z, s, v, _ = run(a, k, q, pi, "full")
    ref = lanczos.block_lanczos(a, k, q, pi)
    check_values(s, ref, 1e-10)
    check_vectors(a, z, s, v, k, EPS[np.float64])


def test_q_capped_returns_warning_and_exact_values():
    sig = 1.0 / np.arange(1, 49)
    a, _, _ = synth.planted(64, 48, sig, 5)
    z, s, st = bk.block_lanczos(dev(a), 16, 4, pi=dev(synth.gaussian_pi(2, 48, 16, np.float64)), stats=True)
    assert st["q_eff"] == 2 and st["width"] == 48
    assert np.allclose(host(s), sig[:16], rtol=1e-10)


# ------------------------------------------------------------------ FP32
@pytest.mark.parametrize("reorth,k,q", [("full", 20, 8), ("full", 10, 6), ("full", 12, 4),
                                         ("local", 20, 4), ("local", 10, 6), ("local", 12, 4)])
def test_fp32_noisy_2000x800(reorth, k, q):
    """k = 20 and 12 (multiples of 4) run the local window on the tensor-core
    orthonormalisation; k = 10 takes the CUDA-core kernels for it.  Local cases stop
    before FP32 rounding has grown into a loss of orthogonality (next test)."""
    a, _ = synth.dense_planted_noisy(n=2000, d=800, rank=200, seed=1002)
    pi = synth.gaussian_pi(2, 800, k)
    z, s, v, st = run(a, k, q, pi, reorth)
    full = lanczos.block_lanczos(a.astype(np.float64), k, q, pi.astype(np.float64), reorth="full")
    check_values(s, full, 1e-5)
    a64 = a.astype(np.float64)
    sig = metrics.true_singular_values(a64)
    r_gpu = metrics.ratios(a64, z, k, sigma=sig)
    r_ora = metrics.ratios(a64, full.Z, k, sigma=sig)
    if reorth == "full":
        check_vectors(a, z, s, v, k, EPS[np.float32])
        for key in r_gpu:
            assert abs(r_gpu[key] - r_ora[key]) <= 1e-3, key


def test_fp32_local_reorthogonalisation_breaks_down_at_q8():
    """The instability Sec. 4 warns of, in FP32: at k = 20, q = 8 on the noisy 2000 x 800
    matrix, reorthogonalising against the two previous blocks only lets the basis lose
    orthogonality completely (an FP32 restatement of the recurrence on the CPU does the
    same), and converged Ritz values reappear as spurious copies that push true ones out
    of the top k.  Full reorthogonalisation on the same input stays accurate."""
    a, _ = synth.dense_planted_noisy(n=2000, d=800, rank=200, seed=1002)
    k, q = 20, 8
    pi = synth.gaussian_pi(2, 800, k)
    full = lanczos.block_lanczos(a.astype(np.float64), k, q, pi.astype(np.float64))
    _, s_full, _, _ = run(a, k, q, pi, "full")
    _, s_loc, _, _ = run(a, k, q, pi, "local")
    check_values(s_full, full, 1e-5)
    assert np.max(np.abs(s_loc - full.sigma) / full.sigma) > 1e-2


def test_fp32_same_results_as_block_krylov():
    """With full reorthogonalisation the basis is Algorithm 2's: the same Ritz values and
    vectors as bks_block_krylov, from a T formed from its band alone."""
    a, _ = synth.dense_planted_noisy(n=4000, d=1500, rank=300, seed=11)
    k, q = 24, 6
    pi = dev(synth.gaussian_pi(5, 1500, k))
    ad = dev(a)
    zl, sl = bk.block_lanczos(ad, k, q, pi=pi)
    zb, sb = bk.block_krylov(ad, k, q, pi=pi)
    zl, sl, zb, sb = host(zl), host(sl), host(zb), host(sb)
    assert np.max(np.abs(sl - sb) / sb) <= 1e-5
    assert metrics.subspace_distance(zl[:, :10], zb[:, :10]) < 1e-3


def test_fp32_cuda_core_path():
    """product_path = SIMT: the band Grams and the three-term update on the CUDA cores."""
    a, _ = synth.dense_planted_noisy(n=2000, d=800, rank=200, seed=1002)
    k, q = 20, 4
    pi = synth.gaussian_pi(2, 800, k)
    z, s, v, _ = run(a, k, q, pi, "full", simt=True)
    full = lanczos.block_lanczos(a.astype(np.float64), k, q, pi.astype(np.float64))
    check_values(s, full, 1e-5)
    check_vectors(a, z, s, v, k, EPS[np.float32])


@pytest.mark.parametrize("q", [1, 2])
def test_fp32_bare_recurrence_at_small_q(q):
    a, _ = synth.dense_planted_noisy(n=2000, d=800, rank=200, seed=1002)
    k = 20
    pi = synth.gaussian_pi(2, 800, k)
    z, s, v, _ = run(a, k, q, pi, "none")
    ref = lanczos.block_lanczos(a.astype(np.float64), k, q, pi.astype(np.float64), reorth="none")
    check_values(s, ref, 1e-5)
    check_vectors(a, z, s, v, k, EPS[np.float32])


# ------------------------------------------------------------------ CSR and BF16
def test_sparse_centred_parity():
    n, d, k, q = 3000, 1500, 20, 8
    row_ptr, col_idx, vals, d = synth.zipf_idf_csr(n=n, d=d, per_row=30, seed=9)
    mu = synth.column_means(row_ptr, col_idx, vals, n, d)
    a = bk.CsrMatrix(dev(row_ptr), dev(col_idx), dev(vals), (n, d), col_mean=dev(mu))
    pi = synth.gaussian_pi(3, d, k)
    z, s = bk.block_lanczos(a, k, q, pi=dev(pi))
    z, s = host(z), host(s)
    op = krylov.centred_csr_op(row_ptr, col_idx, vals, n, d, mu)
    ref = lanczos.block_lanczos(op, k, q, pi)
    check_values(s, ref, 1e-5)
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 1e-5


@pytest.mark.parametrize("form", ["bf16_refined", "bf16_plain"])
def test_bf16_parity(form):
    a = synth.dense_bf16_planted_torch(m=2048, d=1024, seed=2089, device="cuda")
    a64 = a.float().cpu().numpy().astype(np.float64)
    k, q = 20, 4
    pi = synth.gaussian_pi(4, 1024, k)
    ref = lanczos.block_lanczos(a64, k, q, pi)
    kw = dict(precision="bf16", refine=form == "bf16_refined")
    z, s = bk.block_lanczos(a, k, q, pi=dev(pi), **kw)
    z, s = host(z), host(s)
    check_values(s, ref, 1e-5 if form == "bf16_refined" else 3e-4)
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 1e-5


# ------------------------------------------------------------------ arguments
def test_invalid_reorth_mode_is_rejected():
    a = dev(np.ones((10, 5), np.float32))
    lib = bk._binding.load()
    ctx = bk.context(a.device)
    m = bk.dense_matrix(a)
    z = torch.empty((10, 2), device="cuda")
    s = torch.empty((2,), device="cuda")
    import ctypes
    st = lib.bks_block_lanczos(ctx.ptr, ctypes.byref(m), 2, 1, 7, 0, None, ctypes.c_void_p(z.data_ptr()),
                               ctypes.c_void_p(s.data_ptr()), None, None, None)
    assert st == 1   # BKS_ERR_INVALID_ARG, nothing launched
    with pytest.raises(ValueError):
        bk.block_lanczos(a, 2, 1, reorth="partial")
    with pytest.raises(bk.BksError) as e:
        bk.block_lanczos(a, 6, 1)
    assert e.value.status == 1


def test_fp32_full_size_20000x8000_against_block_krylov_and_oracle():
    """The headline workload (20000 x 8000, k = 50, q = 8, width 450) with full
    reorthogonalisation: Ritz values within 1e-5 of the FP64 Algorithm 2 oracle (the same
    space in exact arithmetic) and orthonormal Ritz vectors."""
    a, _ = synth.dense_planted_noisy()
    k, q = 50, 8
    pi = synth.gaussian_pi(2, 8000, k)
    z, s = bk.block_lanczos(dev(a), k, q, pi=dev(pi))
    z, s = host(z), host(s)
    ref = krylov.block_krylov(a.astype(np.float64), k, q, pi.astype(np.float64))
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= 1e-5
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 1e-5
