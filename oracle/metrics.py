"""Error measures of the paper, in FP64 (test infrastructure only).

* Frobenius norm error, eq. (1):  ||A - Z Z^T A||_F / ||A - A_k||_F
* Spectral norm error, eq. (2):   ||A - Z Z^T A||_2 / sigma_{k+1}
* Per-vector error, eq. (3):      max_i |sigma_i^2 - z_i^T A A^T z_i| / sigma_{k+1}^2,
  reported as 1 + that value so all three read as (1 + eps) ratios (Sec. 7 plots the
  maximum deviation over the top k vectors relative to sigma_{k+1}^2).
"""
from __future__ import annotations

import numpy as np


def true_singular_values(a) -> np.ndarray:
    """All singular values of a dense matrix, descending (LAPACK gesdd)."""
    return np.linalg.svd(np.asarray(a, dtype=np.float64), compute_uv=False)


def ratios(a, z, k: int, sigma=None) -> dict:
    """The three (1 + eps) ratios of Z against A.  ``sigma`` holds A's singular values
    (descending, at least k+1 of them, all of them for the Frobenius ratio); they are
    computed with LAPACK when omitted."""
    a64 = np.asarray(a, dtype=np.float64)
    z64 = np.asarray(z, dtype=np.float64)[:, :k]
    if sigma is None:
        sigma = true_singular_values(a64)
    sigma = np.asarray(sigma, dtype=np.float64)
    zta = z64.T @ a64
    resid = a64 - z64 @ zta
    spec = np.linalg.norm(resid, 2)
    frob = np.linalg.norm(resid, "fro")
    tail = np.sqrt(np.sum(sigma[k:] ** 2))
    s_k1 = sigma[k]
    captured = np.einsum("ij,ij->i", zta, zta)          # z_i^T A A^T z_i
    per_vec = np.max(np.abs(sigma[:k] ** 2 - captured)) / s_k1 ** 2
    return {"spectral": spec / s_k1, "frobenius": frob / tail, "per_vector": 1.0 + per_vec}


def captured_energy(a, z) -> np.ndarray:
    """Cumulative ||Z_l^T A||_F^2 for l = 1..k (the quantity Lemma 4.1 maximises)."""
    zta = np.asarray(z, dtype=np.float64).T @ np.asarray(a, dtype=np.float64)
    return np.cumsum(np.einsum("ij,ij->i", zta, zta))


def subspace_distance(z1, z2) -> float:
    """Spectral norm of the difference of the orthogonal projectors onto span(z1), span(z2)."""
    p1 = z1 @ z1.T
    p2 = z2 @ z2.T
    return float(np.linalg.norm(p1 - p2, 2))
