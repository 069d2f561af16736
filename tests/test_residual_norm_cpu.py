"""The residual-norm estimator the full-size parity tests use, pinned on the CPU against
LAPACK's spectral norm (numpy.linalg.norm(., 2), an SVD) on a matrix small enough to
decompose, with the slowly decaying spectrum (sigma_i = i^-1/2) of the BF16 workload,
where the top of the residual spectrum is most clustered."""
import numpy as np
import pytest

import synth
from residual_norm import residual_spectral_norm

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("perturb", [0.0, 1e-3, 1e-1])
def test_estimator_matches_lapack_norm(perturb):
    n, d, k = 1500, 1000, 20
    sigma = np.arange(1, d + 1, dtype=np.float64) ** -0.5
    a, u, _ = synth.planted(n, d, sigma, seed=77)
    rng = np.random.default_rng(5)
    z, _ = np.linalg.qr(u[:, :k] + perturb * rng.standard_normal((n, k)))
    exact = np.linalg.norm(a - z @ (z.T @ a), 2)
    est = residual_spectral_norm(torch.from_numpy(a), torch.from_numpy(z))
    assert est <= exact * (1 + 1e-12)
    assert (exact - est) / exact <= 1e-5, (est, exact)
