"""GPU parity of the block-size-p variant (Sec. 8, "Improved Convergence With Spectral
Decay"): Pi with p >= k columns, every Krylov block p wide, the k leading Ritz vectors
returned; against the FP64 oracle run with the same p-column Pi.

Tolerances as for the p = k path: Ritz values relative 1e-10 (FP64) / 1e-5 (FP32),
orthonormality 100 sqrt(n) eps, subspaces of separated leading groups 1e-8 / 1e-3."""
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
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("method", ["bki", "si"])
def test_block_p_matches_oracle(dtype, method):
    a, sig, _, _ = synth.dense_planted_small()
    a = a.astype(dtype)
    k, p, q = 10, 16, 4
    pi = synth.gaussian_pi(6, 300, p).astype(dtype)
    fn = bk.block_krylov if method == "bki" else bk.simul_iter
    ofn = krylov.block_krylov if method == "bki" else krylov.simul_iter
    z, s, v, st = fn(dev(a), k, q, pi=dev(pi), want_v=True, stats=True, block_p=p)
    z, s, v = host(z), host(s), host(v)
    assert z.shape == (500, k) and s.shape == (k,) and v.shape == (300, k)
    assert st["width"] == (p * (q + 1) if method == "bki" else p)
    ref = ofn(a.astype(np.float64), k, q, pi.astype(np.float64))
    tol = 1e-10 if dtype == np.float64 else 1e-5
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= tol
    eps = EPS[dtype]
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 100 * np.sqrt(500) * eps + 1e-12
    assert metrics.subspace_distance(z[:, :5], ref.Z[:, :5]) < (1e-8 if dtype == np.float64 else 1e-3)
    # a wider block never loses Ritz value against p = k on the same leading columns
    s_k = host(fn(dev(a), k, q, pi=dev(np.ascontiguousarray(pi[:, :k])))[1])
    assert np.all(s >= s_k * (1 - tol))


def test_block_p_seeded_start_matches_oracle_generator():
    a, _, _, _ = synth.dense_planted_small()
    k, p, q = 8, 12, 3
    z, s = bk.block_krylov(dev(a), k, q, seed=77, block_p=p)
    ref = krylov.block_krylov(a, k, q, orng.start_block(77, 300, p))
    assert np.max(np.abs(host(s) - ref.sigma) / ref.sigma) < 1e-6


def test_block_p_caps_q_with_p():
    sig = 1.0 / np.arange(1, 49)
    a, _, _ = synth.planted(64, 48, sig, 5)
    z, s, st = bk.block_krylov(dev(a), 8, 4, pi=dev(synth.gaussian_pi(2, 48, 16, np.float64)), stats=True,
                               block_p=16)
    assert st["q_eff"] == 2 and st["width"] == 48
    assert np.allclose(host(s), sig[:8], rtol=1e-10)


def test_block_p_centred_csr_matches_oracle():
    n, d, k, p, q = 3000, 1000, 6, 12, 3
    row_ptr, col_idx, vals, d = synth.zipf_idf_csr(n=n, d=d, per_row=20, seed=17)
    mu = synth.column_means(row_ptr, col_idx, vals, n, d)
    a = bk.CsrMatrix(dev(row_ptr), dev(col_idx), dev(vals), (n, d), col_mean=dev(mu))
    pi = synth.gaussian_pi(7, d, p)
    z, s = bk.block_krylov(a, k, q, pi=dev(pi), block_p=p)
    op = krylov.centred_csr_op(row_ptr, col_idx, vals, n, d, mu)
    ref = krylov.block_krylov(op, k, q, pi.astype(np.float64))
    assert np.max(np.abs(host(s) - ref.sigma) / ref.sigma) <= 1e-5


def test_block_p_bf16_refined_matches_fp32_form():
    a = synth.dense_bf16_planted_torch(m=4096, d=2048, seed=9, device="cuda")
    k, p, q = 16, 32, 3
    pi = dev(synth.gaussian_pi(8, 2048, p))
    z16, s16 = bk.block_krylov(a, k, q, pi=pi, precision="bf16", block_p=p)
    z32, s32 = bk.block_krylov(a.float().contiguous(), k, q, pi=pi, block_p=p)
    assert np.max(np.abs(host(s16) - host(s32)) / host(s32)) < 1e-5


def test_block_p_batched_equals_single_solves():
    mats = synth.batched_planted(batch=6, k=8, seed=44, m_range=(200, 400), n_range=(150, 300))
    ams = [dev(m) for m in mats]
    outs = bk.block_krylov_batched(ams, 8, 2, seeds=list(range(6)), block_p=12)
    sms = bk.batch_budget(ams, 8, 2)
    for i, (z, s) in enumerate(outs):
        z1, s1 = bk.block_krylov(ams[i], 8, 2, seed=i, block_p=12, max_sms=sms)
        assert torch.equal(z, z1) and torch.equal(s, s1)


def test_block_p_invalid_values_rejected():
    a = dev(np.random.default_rng(0).standard_normal((60, 40)).astype(np.float32))
    for bad in (4, 41, 200):
        with pytest.raises(bk.BksError):
            bk.block_krylov(a, 5, 1, block_p=bad)
    with pytest.raises(bk.BksError):
        bk.ritz_triplets(a, 5, 1, block_p=8)
