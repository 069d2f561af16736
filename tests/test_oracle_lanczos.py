"""Pins of the Block Lanczos oracle (oracle/lanczos.py) against facts other than itself:
the Krylov space and Ritz values of Algorithm 2 (in exact arithmetic the recurrence spans
the same space, Sec. 4), the definition T = Q^T A A^T Q, the three-term property (blocks of
Q^T A A^T Q off the tridiagonal band vanish), orthonormality, the explicit Krylov matrix,
and the (1 + eps) guarantees of eqs. (1)-(3).  The recurrence without reorthogonalisation
is shown to lose orthogonality, the instability the paper warns of."""
import numpy as np
import pytest

import synth
from oracle import krylov, lanczos, metrics


def planted(n=500, d=300, seed=1001):
    a, sig, _, _ = synth.dense_planted_small(n=n, d=d, seed=seed)
    return a, sig


def projector_dist(x, y):
    return metrics.subspace_distance(x, y)


@pytest.mark.parametrize("q", [1, 3, 6])
def test_same_space_and_ritz_values_as_block_krylov(q):
    a, _ = planted()
    k = 10
    pi = synth.gaussian_pi(1, 300, k, dtype=np.float64)
    lz = lanczos.block_lanczos(a, k, q, pi)
    bki = krylov.block_krylov(a, k, q, pi)
    w = k * (q + 1)
    assert lz.Q.shape == (500, w)
    # span(Q_Lanczos) = span(Q_BKI)
    resid = lz.Q - bki.Q @ (bki.Q.T @ lz.Q)
    assert np.linalg.norm(resid, 2) < 1e-10
    # every Ritz value of T equals the one of M = B^T B
    assert np.max(np.abs(lz.lam - bki.lam) / bki.lam[0]) < 1e-12
    assert np.max(np.abs(lz.sigma - bki.sigma) / bki.sigma) < 1e-10
    assert projector_dist(lz.Z[:, :5], bki.Z[:, :5]) < 1e-8


def test_t_is_the_block_tridiagonal_rayleigh_quotient():
    a, _ = planted()
    k, q = 8, 5
    pi = synth.gaussian_pi(3, 300, k, dtype=np.float64)
    lz = lanczos.block_lanczos(a, k, q, pi)
    scale = np.linalg.norm(a, 2) ** 2
    g = lz.Q.T @ a @ (a.T @ lz.Q)   # Q^T A A^T Q straight from the definition
    assert np.max(np.abs(lz.T - g)) < 1e-12 * scale
    w = k * (q + 1)
    band = np.zeros((w, w), dtype=bool)
    for i in range(q + 1):
        for j in range(max(0, i - 1), min(q + 1, i + 2)):
            band[i * k:(i + 1) * k, j * k:(j + 1) * k] = True
    assert np.max(np.abs(g[~band])) < 1e-12 * scale          # the three-term property
    assert np.max(np.abs(lz.Q.T @ lz.Q - np.eye(w))) < 1e-13
    # the sub-diagonal blocks are upper triangular (the R factors of the QR steps)
    for r in lz.R:
        assert np.allclose(r, np.triu(r))


def test_span_of_the_explicit_krylov_matrix():
    a, _ = planted()
    k, q = 6, 2
    pi = synth.gaussian_pi(4, 300, k, dtype=np.float64)
    lz = lanczos.block_lanczos(a, k, q, pi)
    kmat = krylov.krylov_matrix(a, k, q, pi)
    qk, _ = np.linalg.qr(kmat)
    assert projector_dist(lz.Q, qk) < 1e-8


def test_local_reorthogonalisation_agrees_at_small_q():
    a, _ = planted()
    k, q = 10, 3
    pi = synth.gaussian_pi(5, 300, k, dtype=np.float64)
    full = lanczos.block_lanczos(a, k, q, pi, reorth="full")
    loc = lanczos.block_lanczos(a, k, q, pi, reorth="local")
    assert np.max(np.abs(loc.sigma - full.sigma) / full.sigma) < 1e-9
    assert np.max(np.abs(loc.Q.T @ loc.Q - np.eye(loc.Q.shape[1]))) < 1e-8


@pytest.mark.parametrize("q", [1, 2])
def test_the_bare_recurrence_before_orthogonality_is_lost(q):
    """With no reorthogonalisation at all the basis comes from the three-term recurrence
    alone; at small q (before Ritz values converge) it must reproduce the reorthogonalised
    result.  A wrong sign, a missing term or a transposed R_{i-1} breaks this."""
    a, _ = planted()
    k = 10
    pi = synth.gaussian_pi(5, 300, k, dtype=np.float64)
    full = lanczos.block_lanczos(a, k, q, pi, reorth="full")
    bare = lanczos.block_lanczos(a, k, q, pi, reorth="none")
    assert np.max(np.abs(bare.sigma - full.sigma) / full.sigma) < 1e-12
    assert np.max(np.abs(bare.Q.T @ bare.Q - np.eye(bare.Q.shape[1]))) < 1e-10
    assert np.max(np.abs(bare.T - full.T)) < 1e-10 * full.lam[0]


def test_recurrence_alone_loses_orthogonality():
    """Without reorthogonalisation the computed blocks drift away from orthogonality once
    Ritz values converge (the stability issue of Sec. 4); full reorthogonalisation keeps
    Q orthonormal to rounding."""
    a, _ = planted()
    k, q = 5, 20
    pi = synth.gaussian_pi(6, 300, k, dtype=np.float64)
    none = lanczos.block_lanczos(a, k, q, pi, reorth="none")
    full = lanczos.block_lanczos(a, k, q, pi, reorth="full")
    w = none.Q.shape[1]
    assert np.max(np.abs(none.Q.T @ none.Q - np.eye(w))) > 1e-6
    assert np.max(np.abs(full.Q.T @ full.Q - np.eye(w))) < 1e-12


def test_guarantees_at_eps_001():
    a, sig = planted()
    k, q = 10, 6
    for s in range(5):
        pi = synth.gaussian_pi(10 + s, 300, k, dtype=np.float64)
        lz = lanczos.block_lanczos(a, k, q, pi)
        r = metrics.ratios(a, lz.Z, k, sigma=sig)
        assert r["spectral"] <= 1.01 and r["frobenius"] <= 1.01 and r["per_vector"] <= 1.01, r


def test_q_capped_like_algorithm_2():
    a, _ = planted(n=60, d=40)
    k = 10
    pi = synth.gaussian_pi(7, 40, k, dtype=np.float64)
    lz = lanczos.block_lanczos(a, k, 9, pi)
    assert lz.q_eff == krylov.q_effective(60, 40, k, 9) == 3
    assert lz.T.shape == (40, 40)
