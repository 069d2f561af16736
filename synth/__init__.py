"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *builds inputs*: planted-spectrum dense matrices, a Zipf/idf
term-document CSR matrix, Gaussian start blocks and loss targets.  It holds none
of the Block Krylov / Simultaneous Iteration arithmetic; both the FP64 oracle
and the GPU path receive what it produces, so the two sides see identical
inputs.

The paper's datasets (SNAP/amazon0302, SNAP/email-Enron, 20 Newsgroups; Sec. 7)
are not available here; every generator below is a seeded stand-in with the
shape class of those workloads.  Seeds follow one rule: data seed ``1000 + c``
and start-block seed ``c`` for workload ``c``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_pi", "orthonormal", "planted", "dense_planted_small",
    "dense_planted_noisy", "zipf_idf_csr", "column_means", "dense_bf16_planted",
    "batched_planted", "loss_target", "bf16_round",
]


def gaussian_pi(seed: int, d: int, k: int, dtype=np.float32) -> np.ndarray:
    """Start block Pi ~ N(0,1)^{d x k} (Algorithms 1 and 2, step 1), row-major d x k,
    drawn from numpy's PCG64 and rounded to ``dtype``."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((d, k)).astype(dtype)


def orthonormal(rng: np.random.Generator, n: int, r: int) -> np.ndarray:
    """n x r matrix with orthonormal columns: QR of an i.i.d. Gaussian matrix with
    the signs of diag(R) folded in (a Haar-distributed frame)."""
    g = rng.standard_normal((n, r))
    qm, rm = np.linalg.qr(g)
    return qm * np.sign(np.diag(rm))


def planted(n: int, d: int, sigma, seed: int):
    """A = U diag(sigma) V^T in FP64 with seeded orthonormal U (n x r), V (d x r).
    Returns (A, U, V)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.size
    rng = np.random.default_rng(seed)
    u = orthonormal(rng, n, r)
    v = orthonormal(rng, d, r)
    return (u * sigma) @ v.T, u, v


def dense_planted_small(n=500, d=300, seed=1001):
    """Dense FP64 n x d matrix with sigma_i = 1/i, i = 1..min(n, d) (the 500 x 300 workload)."""
    r = min(n, d)
    sigma = 1.0 / np.arange(1, r + 1, dtype=np.float64)
    a, u, v = planted(n, d, sigma, seed)
    return a, sigma, u, v


def dense_planted_noisy(n=20000, d=8000, rank=200, decay=40.0, noise=1e-3, seed=1002,
                        chunk=4096):
    """Dense FP32 n x d matrix U_r diag(exp(-i/decay)) V_r^T + noise * G with G i.i.d. N(0,1)
    (the 20000 x 8000 workload).  Built in row chunks so host memory stays near 2x the
    FP32 result.  Returns (A32, sigma_planted)."""
    rng = np.random.default_rng(seed)
    sigma = np.exp(-np.arange(1, rank + 1, dtype=np.float64) / decay)
    u = orthonormal(rng, n, rank)
    v = orthonormal(rng, d, rank)
    us = u * sigma
    out = np.empty((n, d), dtype=np.float32)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        blk = us[r0:r1] @ v.T
        blk += noise * rng.standard_normal((r1 - r0, d))
        out[r0:r1] = blk
    return out, sigma


def _zipf_cdf(ncols: int, s: float) -> np.ndarray:
    w = np.arange(1, ncols + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_idf_csr(n=200000, d=60000, per_row=50, s=1.1, seed=1003):
    """Term-document-like CSR matrix (the 200000 x 60000 workload).

    Each row holds exactly ``per_row`` distinct columns drawn Zipf(s) over ranks
    1..d by inverse CDF (a repeated column within a row is redrawn), column index =
    rank - 1, indices sorted within each row.  Values are lognormal(0, 1) scaled by
    idf_j = ln(n / df_j), df_j being the number of rows holding column j.
    Returns (row_ptr int64[n+1], col_idx int32[nnz], vals float32[nnz], d).
    """
    rng = np.random.default_rng(seed)
    cdf = _zipf_cdf(d, s)
    cols = np.searchsorted(cdf, rng.random((n, per_row)), side="right").astype(np.int64)
    np.minimum(cols, d - 1, out=cols)
    # Redraw repeats until every row is duplicate-free.
    for _ in range(10000):
        cols.sort(axis=1)
        dup = np.zeros_like(cols, dtype=bool)
        dup[:, 1:] = cols[:, 1:] == cols[:, :-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        fresh = np.searchsorted(cdf, rng.random(nd), side="right")
        cols[dup] = np.minimum(fresh, d - 1)
    else:  # pragma: no cover - the Zipf head saturates long before this
        raise RuntimeError("could not draw duplicate-free rows")
    cols.sort(axis=1)
    df = np.bincount(cols.ravel(), minlength=d).astype(np.float64)
    idf = np.zeros(d)
    nzc = df > 0
    idf[nzc] = np.log(n / df[nzc])
    vals = rng.lognormal(0.0, 1.0, size=(n, per_row)) * idf[cols]
    row_ptr = np.arange(0, n * per_row + 1, per_row, dtype=np.int64)
    return row_ptr, cols.ravel().astype(np.int32), vals.ravel().astype(np.float32), d


def powerlaw_graph_csr(n=262144, out_a=2.0, max_out=2000, s_in=0.9, seed=1006):
    """Directed graph adjacency as a square binary CSR (the stand-in for the paper's
    SNAP/amazon0302 shape class: 262111 nodes, 1.23e6 edges, power-law degrees).

    Out-degree of node u ~ Zipf(out_a) clipped to [1, max_out]; its targets are drawn
    by inverse CDF from Zipf(s_in) over node ranks, mapped through a seeded permutation
    (so the hubs are spread over the index range); repeated targets and self loops are
    dropped; indices sorted within each row; every value is 1.
    Returns (row_ptr int64[n+1], col_idx int32[nnz], vals float32[nnz], n).
    """
    rng = np.random.default_rng(seed)
    deg = np.minimum(rng.zipf(out_a, size=n), max_out).astype(np.int64)
    perm = rng.permutation(n).astype(np.int64)
    cdf = _zipf_cdf(n, s_in)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    dst = perm[np.minimum(np.searchsorted(cdf, rng.random(src.size), side="right"), n - 1)]
    keep = dst != src
    key = np.unique(src[keep] * n + dst[keep])   # sorted by (row, column), duplicates gone
    rows, cols = key // n, key % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), np.ones(cols.size, dtype=np.float32), n


def column_means(row_ptr, col_idx, vals, n, d) -> np.ndarray:
    """mu_j = (1/n) sum_i A_ij: the column means used for implicit centring (FP32)."""
    s = np.bincount(col_idx, weights=vals.astype(np.float64), minlength=d)
    return (s / n).astype(np.float32)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def _fwht_rows(x: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform along the last axis (length a power of 2)."""
    m = x.shape[-1]
    h = 1
    y = x.copy()
    while h < m:
        y = y.reshape(*y.shape[:-1], m // (2 * h), 2, h)
        a = y[..., 0, :].copy()
        b = y[..., 1, :]
        y[..., 0, :] = a + b
        y[..., 1, :] = a - b
        y = y.reshape(*y.shape[:-3], m)
        h *= 2
    return y


def dense_bf16_planted(m=65536, d=16384, seed=1004, rows=None, chunk=1024):
    """A = U diag(i^{-1/2}) V^T with exactly orthonormal Hadamard-based factors, rounded
    to bfloat16 (the 65536 x 16384 workload; m, d powers of two, d <= m).

    U = m^{-1/2} H_m D_1 restricted to its first d columns, V = d^{-1/2} H_d D_2, with
    seeded +-1 diagonals D_1, D_2.  Row r of A is (md)^{-1/2} H_d (D_2 sigma D_1 h_r)
    with h_r[c] = (-1)^popcount(r & c), so any subset of rows can be generated alone.
    Returns (A as FP32 holding bf16 values, sigma)."""
    rng = np.random.default_rng(seed)
    d1 = rng.choice([-1.0, 1.0], size=m)[:d]
    d2 = rng.choice([-1.0, 1.0], size=d)
    sigma = np.arange(1, d + 1, dtype=np.float64) ** -0.5
    scale = d2 * sigma * d1 / np.sqrt(float(m) * float(d))
    rows = np.arange(m) if rows is None else np.asarray(rows)
    cidx = np.arange(d, dtype=np.int64)
    out = np.empty((rows.size, d), dtype=np.float32)
    for i0 in range(0, rows.size, chunk):
        r = rows[i0:i0 + chunk].astype(np.int64)
        pc = np.bitwise_and(r[:, None], cidx[None, :])
        # parity of popcount
        par = np.zeros_like(pc)
        while np.any(pc):
            par ^= pc & 1
            pc >>= 1
        h = 1.0 - 2.0 * par
        out[i0:i0 + chunk] = _fwht_rows(h * scale).astype(np.float32)
    return bf16_round(out), sigma


def dense_bf16_planted_torch(m=65536, d=16384, seed=1004, rows=None, device="cuda", chunk=4096):
    """dense_bf16_planted computed with torch on `device` (a GPU builds the 65536 x 16384
    matrix in seconds): the same FP64 operations in the same order, so the result is
    bitwise identical.  Returns a torch.bfloat16 tensor (rows x d) on `device`."""
    import torch
    rng = np.random.default_rng(seed)
    d1 = rng.choice([-1.0, 1.0], size=m)[:d]
    d2 = rng.choice([-1.0, 1.0], size=d)
    sigma = np.arange(1, d + 1, dtype=np.float64) ** -0.5
    scale = torch.from_numpy(d2 * sigma * d1 / np.sqrt(float(m) * float(d))).to(device)
    rows = np.arange(m) if rows is None else np.asarray(rows)
    cidx = torch.arange(d, dtype=torch.int64, device=device)
    out = torch.empty((rows.size, d), dtype=torch.bfloat16, device=device)
    for i0 in range(0, rows.size, chunk):
        r = torch.from_numpy(rows[i0:i0 + chunk].astype(np.int64)).to(device)
        pc = torch.bitwise_and(r[:, None], cidx[None, :])
        par = torch.zeros_like(pc)
        while bool(torch.any(pc)):
            par ^= pc & 1
            pc >>= 1
        y = (1.0 - 2.0 * par.to(torch.float64)) * scale
        h = 1
        while h < d:   # the butterflies of _fwht_rows, same order
            y = y.reshape(y.shape[0], d // (2 * h), 2, h)
            a = y[:, :, 0, :].clone()
            b = y[:, :, 1, :]
            y[:, :, 0, :] = a + b
            y[:, :, 1, :] = a - b
            y = y.reshape(y.shape[0], d)
            h *= 2
        out[i0:i0 + chunk] = y.to(torch.float32).to(torch.bfloat16)
    return out


def batched_planted(batch=256, k=16, seed=1005, m_range=(256, 4096), n_range=(128, 2048),
                    noise=1e-3):
    """List of dense FP32 matrices with m ~ U[256, 4096], n ~ U[128, 2048] integer shapes,
    each U diag(1/i) V^T + noise * N(0,1) (the batched workload)."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(m_range[0], m_range[1] + 1, size=batch)
    ns = rng.integers(n_range[0], n_range[1] + 1, size=batch)
    out = []
    for b in range(batch):
        m, n = int(ms[b]), int(ns[b])
        r = min(m, n)
        sig = 1.0 / np.arange(1, r + 1, dtype=np.float64)
        u = orthonormal(rng, m, r)
        v = orthonormal(rng, n, r)
        a = (u * sig) @ v.T + noise * rng.standard_normal((m, n))
        out.append(a.astype(np.float32))
    return out


def loss_target(seed: int, n: int, d: int, dtype=np.float64) -> np.ndarray:
    """T ~ N(0,1)^{n x d}: the target of the loss sum(Sigma_k) + ||A_k - T||_F^2."""
    return np.random.default_rng(seed).standard_normal((n, d)).astype(dtype)
