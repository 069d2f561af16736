"""Exact adjoint of Sigma_k and A_k = U_k U_k^T A through a full SVD, in FP64
(test infrastructure only).

The paper does not differentiate its outputs; this is the reference the GPU
backward is held to.  With A = U diag(s) V^T (thin, r = min(n, d) triplets),
upstream gradients g (k-vector, for Sigma_k) and G (n x d, for A_k),
P = U_k U_k^T and lambda = s^2:

  dL/dA = U_k diag(g) V_k^T + P G
          + sum_{i <= k < j <= r} c_ij (s_i u_j v_i^T + s_j u_i v_j^T)
          + (I - U U^T) G V_k V_k^T,
  c_ij  = (s_i u_j^T G v_i + s_j u_i^T G v_j) / (lambda_i - lambda_j).

The first two terms are the direct parts; the pair sum is the rotation of the
top-k subspace toward triplet j; the last term is its rotation toward the part of
R^n outside range(U).  Pairs inside the top k do not appear because A_k depends
on U_k only through its span.  ``central_difference`` pins the formula.
"""
from __future__ import annotations

import numpy as np


def truncated(a, k):
    """(U_k, s, V_k, A_k) from LAPACK's SVD."""
    u, s, vt = np.linalg.svd(np.asarray(a, dtype=np.float64), full_matrices=False)
    ak = (u[:, :k] * s[:k]) @ vt[:k]
    return u, s, vt.T, ak


def loss(a, k, t):
    """L(A) = sum(Sigma_k) + ||A_k - T||_F^2."""
    _, s, _, ak = truncated(a, k)
    return float(s[:k].sum() + np.sum((ak - t) ** 2))


def adjoint_from_triplets(u, s, v, k, g_sigma, g_ak, gap_tau=0.0):
    """The formula above with the given triplets (u: n x r, s: r descending, v: d x r) in
    place of a full SVD; (I - U U^T) then projects out the span of the given u.  It is the
    exact gradient when the triplets span range(A) (e.g. A of rank <= r).  With gap_tau > 0,
    c_ij is taken as 0 where lambda_i - lambda_j <= gap_tau lambda_1 (near-degenerate pairs)."""
    u, s, v = (np.asarray(x, dtype=np.float64) for x in (u, s, v))
    g_sigma = np.asarray(g_sigma, dtype=np.float64)
    uk, vk = u[:, :k], v[:, :k]
    out = (uk * g_sigma) @ vk.T
    if g_ak is None:
        return out
    g = np.asarray(g_ak, dtype=np.float64)
    out += uk @ (uk.T @ g)
    utgv = u.T @ g @ v                               # (r x r): entry (a, b) = u_a^T G v_b
    si = s[:k][:, None]
    sj = s[k:][None, :]
    lam_gap = si ** 2 - sj ** 2
    keep = lam_gap > gap_tau * s[0] ** 2
    c = np.where(keep, (si * utgv[k:, :k].T + sj * utgv[:k, k:]) / np.where(keep, lam_gap, 1.0), 0.0)
    out += u[:, k:] @ (c.T * s[:k][None, :]) @ vk.T
    out += uk @ (c * s[k:][None, :]) @ v[:, k:].T
    out += (g @ vk - u @ (u.T @ (g @ vk))) @ vk.T
    return out


def adjoint(a, k, g_sigma, g_ak):
    """dL/dA for upstream gradients g_sigma (k) and g_ak (n x d, or None), through LAPACK's
    full thin SVD of A."""
    u, s, v, _ = truncated(a, k)
    return adjoint_from_triplets(u, s, v, k, g_sigma, g_ak)


def loss_grad(a, k, t):
    """Gradient of L(A) = sum(Sigma_k) + ||A_k - T||_F^2."""
    _, _, _, ak = truncated(a, k)
    return adjoint(a, k, np.ones(k), 2.0 * (ak - np.asarray(t, dtype=np.float64)))


def central_difference(a, k, t, h=None):
    """Central finite differences of L over every entry of A (small matrices only).

    L(A+) - L(A-) is formed as (sum s+ - sum s-) + <A_k+ - A_k-, (A_k+ - T) + (A_k- - T)>,
    which equals the plain difference exactly (|X|^2 - |Y|^2 = <X - Y, X + Y>) but does
    not subtract two nearly equal loss values of size ||T||_F^2."""
    a64 = np.array(a, dtype=np.float64, copy=True)
    t64 = np.asarray(t, dtype=np.float64)
    if h is None:
        h = 1e-6 * float(np.max(np.abs(a64)))
    out = np.empty_like(a64)
    for i in range(a64.shape[0]):
        for j in range(a64.shape[1]):
            old = a64[i, j]
            a64[i, j] = old + h
            _, sp, _, akp = truncated(a64, k)
            a64[i, j] = old - h
            _, sm, _, akm = truncated(a64, k)
            a64[i, j] = old
            diff = (sp[:k] - sm[:k]).sum() + np.sum((akp - akm) * ((akp - t64) + (akm - t64)))
            out[i, j] = diff / (2 * h)
    return out
