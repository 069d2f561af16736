"""Seeded input generators: properties of the synthetic workloads (no GPU)."""
import numpy as np
import pytest

import synth


def test_bf16_planted_torch_matches_numpy_bitwise():
    torch = pytest.importorskip("torch")
    rows = np.array([0, 1, 5, 77, 1000, 2047, 4095])
    a, _ = synth.dense_bf16_planted(m=4096, d=1024, rows=rows)
    b = synth.dense_bf16_planted_torch(m=4096, d=1024, rows=rows, device="cpu")
    assert b.dtype == torch.bfloat16
    assert np.array_equal(a.view(np.uint32), b.float().numpy().view(np.uint32))


def test_bf16_planted_spectrum():
    """Before rounding the factors are exactly orthonormal: the singular values of the
    BF16 matrix sit within the rounding perturbation of sigma_i = i^{-1/2}."""
    a, sigma = synth.dense_bf16_planted(m=1024, d=256)
    s = np.linalg.svd(a.astype(np.float64), compute_uv=False)
    # |E|_2 <= |E|_F <= 2^-9 |A|_F for round-to-nearest BF16
    bound = 2.0 ** -9 * np.linalg.norm(a.astype(np.float64))
    assert np.max(np.abs(s - sigma)) <= bound
    assert np.array_equal(a, synth.bf16_round(a))


def test_bf16_round_ties_to_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5], np.float32)
    r = synth.bf16_round(x)
    assert r.tolist() == [1.0, 1.0, 1.0 + 2 * 2.0 ** -7, 1.0, -2.5]


def test_powerlaw_graph_structure():
    """The directed power-law graph stand-in: square, binary, sorted duplicate-free rows
    without self loops, seeded, and amazon0302-sized at the defaults (262111 nodes,
    1.23e6 edges: within 15%)."""
    rp, ci, cv, n = synth.powerlaw_graph_csr(n=20000, seed=3)
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 0)
    assert np.all(cv == 1.0) and ci.min() >= 0 and ci.max() < n
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(ci != rows)
    same_row = rows[1:] == rows[:-1]
    assert np.all(ci[1:][same_row] > ci[:-1][same_row])
    rp2, ci2, _, _ = synth.powerlaw_graph_csr(n=20000, seed=3)
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
    # heavy tails on both sides: the largest in-degree is far above the mean
    indeg = np.bincount(ci, minlength=n)
    assert indeg.max() > 50 * ci.size / n
    rp, ci, _, n = synth.powerlaw_graph_csr()
    assert n == 262144 and abs(ci.size - 1.23e6) < 0.15 * 1.23e6
