"""Block Lanczos, the classic relative of Algorithm 2 (Sec. 4, "computing Q"), in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper notes that the traditional Block Lanczos algorithm builds the basis of the same
Krylov space of A A^T, started from an orthonormal basis Q_0 of A Pi, by a three-term
recurrence that makes Q^T A A^T Q block tridiagonal with k x k blocks, which is cheaper to
decompose when qk is large, and that the recurrence can need extra steps to keep Q
orthogonal.  Written out (with D_i the diagonal and R_i the sub-diagonal blocks):

    A A^T Q_i = Q_{i-1} R_{i-1}^T + Q_i D_i + Q_{i+1} R_i,     D_i = Q_i^T A A^T Q_i,

i.e. W_i = A A^T Q_i - Q_i D_i - Q_{i-1} R_{i-1}^T is factorised as W_i = Q_{i+1} R_i, and

    T = [[D_0, R_0^T,       ],
         [R_0, D_1,   R_1^T ],
         [     R_1,   D_2, ..]]   (w x w, w = k (q + 1)).

The extra steps (the reading taken here) are a reorthogonalisation of W_i before its QR:
"full" projects it twice against every earlier block, "local" twice against Q_i and
Q_{i-1} only (the blocks the recurrence itself uses), "none" not at all.  Rayleigh-Ritz
then takes the eigenvectors of T for its k largest eigenvalues, Z = Q Ubar_k and
Sigma_k = sqrt(lambda_1..k(T)), with the same sign convention as Algorithm 2.  q is capped
as for Algorithm 2 so that w <= min(n, d).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .krylov import _as_op, _start_block, orthonormalise, q_effective


@dataclass
class LanczosResult:
    Z: np.ndarray        # n x k Ritz vectors
    sigma: np.ndarray    # k Ritz values, descending
    Q: np.ndarray        # n x w basis from the recurrence
    B: np.ndarray        # d x w, A^T Q
    T: np.ndarray        # w x w block-tridiagonal Rayleigh quotient
    D: list              # diagonal blocks D_i
    R: list              # sub-diagonal blocks R_i
    lam: np.ndarray      # eigenvalues of T, descending
    Ubar: np.ndarray     # eigenvectors of T in the order of lam
    q_eff: int


def assemble_tridiagonal(d_blocks, r_blocks) -> np.ndarray:
    """The block-tridiagonal T from its diagonal blocks D_i and sub-diagonal blocks R_i."""
    k = d_blocks[0].shape[0]
    nb = len(d_blocks)
    t = np.zeros((nb * k, nb * k))
    for i, di in enumerate(d_blocks):
        t[i * k:(i + 1) * k, i * k:(i + 1) * k] = di
    for i, ri in enumerate(r_blocks):
        t[(i + 1) * k:(i + 2) * k, i * k:(i + 1) * k] = ri
        t[i * k:(i + 1) * k, (i + 1) * k:(i + 2) * k] = ri.T
    return t


def block_lanczos(a, k: int, q: int, pi, reorth: str = "full") -> LanczosResult:
    """Block Lanczos on A A^T from Q_0 = orth(A Pi), q further blocks, Rayleigh-Ritz on T."""
    if reorth not in ("full", "local", "none"):
        raise ValueError("reorth must be 'full', 'local' or 'none'")
    op = _as_op(a)
    pi64 = _start_block(pi, op.d, k)
    p = pi64.shape[1]
    q_eff = q_effective(op.n, op.d, p, q)
    qs = [orthonormalise(op.mul(pi64))]
    bs, d_blocks, r_blocks = [], [], []
    for i in range(q_eff + 1):
        b_i = op.tmul(qs[i])                 # A^T Q_i
        bs.append(b_i)
        u = op.mul(b_i)                      # A A^T Q_i
        d_i = qs[i].T @ u
        d_blocks.append(0.5 * (d_i + d_i.T))
        if i == q_eff:
            break
        w = u - qs[i] @ d_blocks[i]
        if i > 0:
            w = w - qs[i - 1] @ r_blocks[i - 1].T
        if reorth != "none":
            basis = np.hstack(qs if reorth == "full" else qs[max(0, i - 1):])
            for _pass in range(2):
                w = w - basis @ (basis.T @ w)
        q_next, r_i = np.linalg.qr(w, mode="reduced")
        qs.append(q_next)
        r_blocks.append(r_i)
    t = assemble_tridiagonal(d_blocks, r_blocks)
    lam, ub = np.linalg.eigh(t)
    order = np.argsort(-lam, kind="stable")
    lam, ub = lam[order], ub[:, order]
    q_mat = np.hstack(qs)
    z = q_mat @ ub[:, :k]
    idx = np.argmax(np.abs(z), axis=0)
    s = np.sign(z[idx, np.arange(k)])
    s[s == 0] = 1.0
    z = z * s
    ub = ub.copy()
    ub[:, :k] *= s
    return LanczosResult(z, np.sqrt(np.maximum(lam[:k], 0.0)), q_mat, np.hstack(bs), t, d_blocks,
                         r_blocks, lam, ub, q_eff)
