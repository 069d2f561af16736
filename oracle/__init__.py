"""FP64 CPU oracle for randomized Simultaneous Iteration and Block Krylov Iteration.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of Musco & Musco, "Randomized Block Krylov Methods for Stronger and
Faster Approximate Singular Value Decomposition" (arXiv 1504.05477).  Only the
test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it.  The GPU library never calls it and shares no code with it; the only
thing the two sides share is the seeded input generators in ``synth``.

Modules
  krylov   Algorithm 1 (Simultaneous Iteration) and Algorithm 2 (Block Krylov
           Iteration) with per-iteration reorthonormalisation (Sec. 4.1, 4.2) and
           the Rayleigh-Ritz post-processing of Lemma 4.1.
  jacobi   one-sided (Hestenes) Jacobi SVD, used to pin the oracle's eigen-solver.
  metrics  the three error measures of eqs. (1)-(3).
  rng      SplitMix64 + Box-Muller start block, the counter-based generator the
           GPU library also implements (from the published definitions).
  grad     exact adjoint of Sigma_k and A_k through a full SVD, plus central
           finite differences.
  lanczos  Block Lanczos (Sec. 4): the three-term block recurrence with a block-
           tridiagonal Q^T A A^T Q, with full, local or no reorthogonalisation.

Every function here is pinned by ``tests/test_oracle_pins.py`` (and the Block Lanczos
module by ``tests/test_oracle_lanczos.py``) against closed forms, LAPACK, planted
spectra, invariants and the worked example of Sec. 2.2.
"""
from . import krylov, jacobi, metrics, rng, grad, lanczos  # noqa: F401
from .krylov import block_krylov, simul_iter, dense_op, centred_csr_op  # noqa: F401
