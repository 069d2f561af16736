"""Spectral norm of the residual A - Z Z^T A (the numerator of eq. (2), Sec. 1) for
matrices too large for a dense SVD, test infrastructure only.

R = (I - Z Z^T) A is touched only through R X = A X - Z (Z^T A X) and R^T Y = A^T Y
(Y already orthogonal to Z).  A block Krylov space of R^T R (start block X_0 ~ N(0,1),
`block` columns, `iters` further blocks, each re-orthogonalised twice) is built, and
||R||_2 is the largest singular value of R restricted to it (Rayleigh-Ritz), so the
estimate never exceeds the true norm.  Runs in torch on whatever device A lives on;
the Gram of the final block is formed in FP64.
"""
from __future__ import annotations


def residual_spectral_norm(a, z, block=32, iters=20, seed=0, dtype=None):
    import torch
    dt = dtype or (torch.float32 if a.is_cuda else torch.float64)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        a = a.to(dt)
        z = z.to(device=a.device, dtype=dt)
        g = torch.Generator(device="cpu").manual_seed(seed)
        d = a.shape[1]

        def r_mul(x):
            y = a @ x
            return y - z @ (z.T @ y)

        basis = []
        x = torch.randn((d, block), generator=g, dtype=torch.float64).to(device=a.device, dtype=dt)
        for _ in range(iters + 1):
            for _ in range(2):   # block Gram-Schmidt, twice
                for b in basis:
                    x = x - b @ (b.T @ x)
            x, _ = torch.linalg.qr(x)
            basis.append(x)
            x = a.T @ r_mul(x)
        k = torch.cat(basis, dim=1)
        rk = r_mul(k).to(torch.float64)
        lam = torch.linalg.eigvalsh(rk.T @ rk)
        return float(torch.sqrt(torch.clamp(lam[-1], min=0.0)))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
