"""One-sided (Hestenes) Jacobi SVD in FP64 (test infrastructure only).

Used to pin the oracle's eigen-solver: the top singular vectors of M (Algorithms
1 and 2, step 5) must agree with an independent SVD computed by plane rotations.
For a column pair (p, q) with alpha = |x_p|^2, beta = |x_q|^2, gamma = x_p . x_q the
rotation [c s; -s c] with zeta = (beta - alpha) / (2 gamma),
t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t makes the
two columns orthogonal; sweeps repeat until every pair is orthogonal to ``tol``.
"""
from __future__ import annotations

import math

import numpy as np


def jacobi_svd(g, tol: float = 1e-15, max_sweeps: int = 80):
    """Return (U, s, V) with G = U diag(s) V^T, s descending, for an m x n matrix G
    (m >= n).  Columns of U whose singular value is zero are left as zero vectors."""
    x = np.array(g, dtype=np.float64, copy=True)
    m, n = x.shape
    if m < n:
        raise ValueError("jacobi_svd expects m >= n")
    v = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                xp = x[:, p]
                xq = x[:, q]
                alpha = float(xp @ xp)
                beta = float(xq @ xq)
                gamma = float(xp @ xq)
                if gamma == 0.0 or abs(gamma) <= tol * math.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                xp_old = xp.copy()
                x[:, p] = c * xp_old - s * xq
                x[:, q] = s * xp_old + c * xq
                vp_old = v[:, p].copy()
                v[:, p] = c * vp_old - s * v[:, q]
                v[:, q] = s * vp_old + c * v[:, q]
        if not rotated:
            break
    else:
        raise RuntimeError("Jacobi SVD did not converge")
    s = np.sqrt(np.einsum("ij,ij->j", x, x))
    order = np.argsort(-s, kind="stable")
    s = s[order]
    x = x[:, order]
    v = v[:, order]
    u = np.zeros_like(x)
    nz = s > 0
    u[:, nz] = x[:, nz] / s[nz]
    return u, s, v


def jacobi_eigh_psd(m):
    """Eigen-decomposition of a symmetric positive semi-definite matrix through its SVD:
    returns (lam descending, vectors).  For PSD M the singular values are the
    eigenvalues and the right singular vectors are eigenvectors."""
    _, s, v = jacobi_svd(m)
    return s, v
