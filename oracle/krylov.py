"""Algorithms 1 and 2 of the paper, step by step, in FP64 (test infrastructure only).

Notation follows the paper: A is n x d, Pi is the d x k Gaussian start block,
q the iteration count, K the Krylov matrix, Q an orthonormal basis of span(K),
M = Q^T A A^T Q, Ubar_k its top-k eigenvectors and Z = Q Ubar_k.

Readings of the paper taken here (each listed in the design notes):
* BKI keeps q+1 blocks, so Q has w = k(q+1) columns (Alg. 2 step 2; the "qk" of
  steps 3-4 counts the blocks after the first).
* Orthonormalisation happens block by block as K is built (Sec. 4.1 and 4.2: it
  leaves span(K) unchanged in exact arithmetic).  Each new block is A A^T applied
  to the previous *orthonormal* block, projected twice against all earlier blocks,
  then orthonormalised with Householder QR.
* M is formed "left to right" as B^T B with B = A^T Q (Sec. 4.1 and 4.2), reusing
  the products A^T Q_i that also drive the iteration.
* M is symmetric positive semi-definite, so its top singular vectors are its
  eigenvectors for the largest eigenvalues; Sigma_k = sqrt(lambda_1..k).
* When k(q+1) > min(n, d) the Krylov space cannot grow: q is capped at
  q_eff = min(q, floor(min(n, d)/k) - 1).
* Each Ritz vector's sign is fixed so that its entry of largest magnitude is
  positive (lowest index on ties).
* Pi may have p >= k columns (Sec. 8, "Improved Convergence With Spectral Decay"):
  every block then has p columns, w = p(q+1) (q capped with p in place of k), and the
  k leading Ritz vectors are returned.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Operator:
    """A matrix seen only through products with A and A^T (Sec. 4: the methods touch A
    only through these products)."""
    n: int
    d: int
    mul: callable    # X (d x c) -> A X (n x c)
    tmul: callable   # Y (n x c) -> A^T Y (d x c)
    dense: callable  # () -> A as a dense FP64 array (metrics on small cases)


def dense_op(a) -> Operator:
    """Operator for a dense matrix, upcast exactly to FP64."""
    a64 = np.asarray(a, dtype=np.float64)
    return Operator(a64.shape[0], a64.shape[1], lambda x: a64 @ x, lambda y: a64.T @ y,
                    lambda: a64)


def centred_csr_op(row_ptr, col_idx, vals, n, d, mu) -> Operator:
    """Operator for A_c = A - 1 mu^T with A in CSR (FP64 upcast) and mu the column means
    (footnote 1 of Sec. 1: principal components after mean centring).  The centring is
    applied implicitly: A_c X = A X - 1 (mu^T X), A_c^T Y = A^T Y - mu (1^T Y)."""
    import scipy.sparse as sp
    a = sp.csr_matrix((np.asarray(vals, np.float64), np.asarray(col_idx), np.asarray(row_ptr)),
                      shape=(n, d))
    at = a.T.tocsr()
    mu64 = np.asarray(mu, dtype=np.float64) if mu is not None else np.zeros(d)
    ones = np.ones(n)

    def mul(x):
        return a @ x - np.outer(ones, mu64 @ x)

    def tmul(y):
        return at @ y - np.outer(mu64, ones @ y)

    def dense():
        return a.toarray() - np.outer(ones, mu64)

    return Operator(n, d, mul, tmul, dense)


def _as_op(a) -> Operator:
    return a if isinstance(a, Operator) else dense_op(a)


def q_effective(n: int, d: int, k: int, q: int) -> int:
    """Largest usable iteration count: the Krylov width k(q+1) may not exceed min(n, d)."""
    return max(0, min(q, min(n, d) // k - 1))


def orthonormalise(w: np.ndarray) -> np.ndarray:
    """Orthonormal basis of span(W) by Householder QR (Sec. 4.1: Gram-Schmidt or
    Householder reflections), reduced form."""
    qm, _ = np.linalg.qr(w, mode="reduced")
    return qm


def sign_fix(z: np.ndarray) -> np.ndarray:
    """Flip each column so its entry of largest magnitude (lowest index on ties) is positive."""
    idx = np.argmax(np.abs(z), axis=0)
    s = np.sign(z[idx, np.arange(z.shape[1])])
    s[s == 0] = 1.0
    return z * s


@dataclass
class Result:
    Z: np.ndarray        # n x k Ritz vectors, orthonormal columns
    sigma: np.ndarray    # k Ritz values, descending
    Q: np.ndarray        # n x w orthonormal basis of span(K)
    B: np.ndarray        # d x w, B = A^T Q
    M: np.ndarray        # w x w, M = Q^T A A^T Q = B^T B
    lam: np.ndarray      # w eigenvalues of M, descending
    Ubar: np.ndarray     # w x w eigenvectors of M, columns in the order of lam
    q_eff: int


def _rayleigh_ritz(q_mat: np.ndarray, b_mat: np.ndarray, k: int, q_eff: int) -> Result:
    """Steps 4-6 of Algorithms 1 and 2 with Lemma 4.1: M = Q^T A A^T Q = B^T B,
    Ubar_k = top-k eigenvectors of M, Z = Q Ubar_k."""
    m = b_mat.T @ b_mat
    m = 0.5 * (m + m.T)
    lam, ub = np.linalg.eigh(m)
    order = np.argsort(-lam, kind="stable")
    lam = lam[order]
    ub = ub[:, order]
    z = q_mat @ ub[:, :k]
    # make each Ritz vector's largest entry positive; carry the sign into Ubar
    idx = np.argmax(np.abs(z), axis=0)
    s = np.sign(z[idx, np.arange(k)])
    s[s == 0] = 1.0
    z = z * s
    ub = ub.copy()
    ub[:, :k] *= s
    sigma = np.sqrt(np.maximum(lam[:k], 0.0))
    return Result(z, sigma, q_mat, b_mat, m, lam, ub, q_eff)


def _start_block(pi, d: int, k: int) -> np.ndarray:
    """Pi as FP64, d x p with p >= k columns (p = k in Algorithms 1 and 2, any p >= k in
    Sec. 8)."""
    pi64 = np.asarray(pi, dtype=np.float64)
    if pi64.ndim != 2 or pi64.shape[0] != d or pi64.shape[1] < k:
        raise ValueError(f"Pi must be {d} x p with p >= {k}, got {pi64.shape}")
    return pi64


def block_krylov(a, k: int, q: int, pi) -> Result:
    """Algorithm 2 (Block Krylov Iteration), FP64.

    K = [A Pi, (A A^T) A Pi, ..., (A A^T)^q A Pi] is built one block at a time; block
    i is A A^T Q_{i-1}, projected twice against Q_0..Q_{i-1} (block classical
    Gram-Schmidt with reorthogonalisation) and orthonormalised, which spans the same
    space as the paper's explicit K.  B_i = A^T Q_i is kept and M = B^T B.
    """
    op = _as_op(a)
    pi64 = _start_block(pi, op.d, k)
    q_eff = q_effective(op.n, op.d, pi64.shape[1], q)
    qs = [orthonormalise(op.mul(pi64))]
    bs = []
    for _ in range(q_eff):
        b_prev = op.tmul(qs[-1])            # A^T Q_{i-1}
        bs.append(b_prev)
        w = op.mul(b_prev)                  # (A A^T) Q_{i-1}
        q_cat = np.hstack(qs)
        for _pass in range(2):
            w = w - q_cat @ (q_cat.T @ w)
        qs.append(orthonormalise(w))
    bs.append(op.tmul(qs[-1]))               # A^T Q_q
    return _rayleigh_ritz(np.hstack(qs), np.hstack(bs), k, q_eff)


def ritz_values(b_mat: np.ndarray, k: int) -> np.ndarray:
    """The min(k, w) leading Ritz values sqrt(lambda_i(B^T B)) of the space whose kept
    products are the columns of B (Lemma 4.1: M = B^T B)."""
    lam = np.linalg.eigvalsh(b_mat.T @ b_mat)[::-1]
    return np.sqrt(np.maximum(lam[:min(k, lam.size)], 0.0))


def block_krylov_adaptive(a, k: int, q_max: int, tol: float, pi):
    """Algorithm 2 with the iteration count chosen on the fly.  After B_{i-1} = A^T Q_{i-1}
    the k leading Ritz values of the i-block space are compared with those of the
    (i-1)-block space; the first i >= 2 where none moved by more than tol (relative to its
    new value) ends the iteration, and Rayleigh-Ritz runs on those i blocks (q = i - 1).
    Returns (Result, the relative changes observed, in order)."""
    op = _as_op(a)
    pi64 = _start_block(pi, op.d, k)
    q_cap = q_effective(op.n, op.d, pi64.shape[1], q_max)
    qs = [orthonormalise(op.mul(pi64))]
    bs = []
    prev = None
    deltas = []
    for i in range(1, q_cap + 1):
        b_prev = op.tmul(qs[-1])
        bs.append(b_prev)
        cur = ritz_values(np.hstack(bs), k)
        if prev is not None:
            floor = 1e-30 + 1e-12 * cur[0]
            delta = float(np.max(np.abs(cur - prev) / np.maximum(cur, floor)))
            deltas.append(delta)
            if delta <= tol:
                return _rayleigh_ritz(np.hstack(qs), np.hstack(bs), k, i - 1), deltas
        prev = cur
        w = op.mul(b_prev)
        q_cat = np.hstack(qs)
        for _pass in range(2):
            w = w - q_cat @ (q_cat.T @ w)
        qs.append(orthonormalise(w))
    bs.append(op.tmul(qs[-1]))
    return _rayleigh_ritz(np.hstack(qs), np.hstack(bs), k, q_cap), deltas


def simul_iter(a, k: int, q: int, pi) -> Result:
    """Algorithm 1 (Simultaneous Iteration), FP64, orthonormalised after every
    iteration (Sec. 4.1): Q <- orth(A A^T Q), starting from Q = orth(A Pi)."""
    op = _as_op(a)
    pi64 = _start_block(pi, op.d, k)
    qm = orthonormalise(op.mul(pi64))
    for _ in range(q):
        qm = orthonormalise(op.mul(op.tmul(qm)))
    return _rayleigh_ritz(qm, op.tmul(qm), k, q)


def krylov_matrix(a, k: int, q: int, pi) -> np.ndarray:
    """The explicit K = [A Pi, (A A^T) A Pi, ..., (A A^T)^q A Pi] of Algorithm 2 step 2,
    without any orthonormalisation (ill conditioned; only for small-q checks)."""
    op = _as_op(a)
    blk = op.mul(np.asarray(pi, dtype=np.float64))
    out = [blk]
    for _ in range(q):
        blk = op.mul(op.tmul(blk))
        out.append(blk)
    return np.hstack(out)
