"""Pins for the FP64 oracle: every check compares it with something other than itself
(closed forms, LAPACK, planted spectra, exact invariants, the worked example of
Sec. 2.2, finite differences), chosen so that a dropped term, a wrong sign, index
or transposed operand in the oracle fails at least one of them."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import krylov, jacobi, metrics, rng, grad

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _planted(n, d, sigma, seed):
    a, u, v = synth.planted(n, d, sigma, seed)
    return a, u, v


# ---------------------------------------------------------------- Jacobi SVD
def test_jacobi_matches_lapack_random():
    g = np.random.default_rng(0).standard_normal((64, 48))
    u, s, v = jacobi.jacobi_svd(g)
    s_ref = np.linalg.svd(g, compute_uv=False)
    assert np.max(np.abs(s - s_ref) / s_ref) < 1e-13
    assert np.allclose(u @ np.diag(s) @ v.T, g, atol=1e-13)
    assert np.allclose(v.T @ v, np.eye(48), atol=1e-13)
    # leading singular vectors agree with LAPACK's up to sign
    ul, _, _ = np.linalg.svd(g, full_matrices=False)
    for i in range(5):
        assert abs(abs(ul[:, i] @ u[:, i]) - 1) < 1e-10


def test_jacobi_rank_deficient_and_planted():
    sig = np.array([5.0, 3.0, 2.0, 1.0, 0.5, 0.25, 0.125, 0.0625, 0.03, 0.01])
    a, uu, vv = _planted(40, 30, sig, 7)
    _, s, _ = jacobi.jacobi_svd(a)
    assert np.allclose(s[:10], sig, rtol=1e-12)
    assert np.all(s[10:] < 1e-13)


def test_jacobi_eigh_psd_matches_closed_form():
    lam = np.array([9.0, 4.0, 1.0, 0.25])
    qm = np.linalg.qr(np.random.default_rng(3).standard_normal((4, 4)))[0]
    m = (qm * lam) @ qm.T
    l_j, v_j = jacobi.jacobi_eigh_psd(m)
    assert np.allclose(l_j, lam, rtol=1e-13)
    assert np.allclose(np.abs(np.sum(v_j * qm, axis=0)), 1.0, atol=1e-12)


# ---------------------------------------------------------- exactness cases
def test_block_krylov_exact_when_width_covers_rank():
    # 60 x 40, rank 40, k = 10, q = 3: w = 40 spans range(A), so Z = U_k exactly.
    sig = 1.0 / np.arange(1, 41)
    a, u, v = _planted(60, 40, sig, 11)
    pi = synth.gaussian_pi(1, 40, 10)
    res = krylov.block_krylov(a, 10, 3, pi)
    assert res.q_eff == 3 and res.Q.shape == (60, 40)
    assert np.max(np.abs(res.sigma - sig[:10]) / sig[:10]) < 1e-12
    assert metrics.subspace_distance(res.Z, u[:, :10]) < 1e-10
    for i in range(10):
        assert abs(abs(res.Z[:, i] @ u[:, i]) - 1) < 1e-10


# ------------------------------------------- block size p >= k (Sec. 8, spectral decay)
def test_block_p_exact_when_first_block_covers_rank():
    # rank 20, k = 5, p = 20, q = 0: span(A Pi) = range(A), so Z = U_5 and sigma exact
    sig = np.concatenate([1.0 / np.arange(1, 21), np.zeros(20)])
    a, u, v = _planted(60, 40, sig, 12)
    pi = synth.gaussian_pi(3, 40, 20, np.float64)
    for fn in (krylov.block_krylov, krylov.simul_iter):
        res = fn(a, 5, 0, pi)
        assert res.Q.shape == (60, 20) and res.Z.shape == (60, 5)
        assert np.max(np.abs(res.sigma - sig[:5]) / sig[:5]) < 1e-12
        assert metrics.subspace_distance(res.Z, u[:, :5]) < 1e-10


@pytest.mark.parametrize("fn", [krylov.block_krylov, krylov.simul_iter])
def test_block_p_ritz_values_dominate_block_k(fn):
    # Pi_p = [Pi_k, more columns]: span(Q_p) contains span(Q_k), so by Courant-Fischer
    # every one of the k leading Ritz values can only grow
    a, _ = synth.dense_planted_noisy(n=800, d=500, rank=100, seed=4)
    pi = synth.gaussian_pi(5, 500, 16, np.float64)
    for q in (0, 1, 3):
        rk = fn(a, 8, q, pi[:, :8])
        rp = fn(a, 8, q, pi)
        assert np.all(rp.sigma >= rk.sigma - 1e-12 * rk.sigma[0])


def test_block_p_gap_dependent_convergence():
    # Theorem "Gap Dependent Convergence": with sigma_k / sigma_{k+1} - 1 ~ 1e-3 but
    # sigma_k / sigma_{p+1} = 2, p = 20 reaches the per-vector and spectral guarantees
    # at q = 2 where p = k = 10 does not
    sig = np.concatenate([np.linspace(1.0, 0.9, 10), np.linspace(0.899, 0.88, 10),
                          0.45 * np.exp(-np.arange(380) / 30)])
    a, u, v = _planted(600, 400, sig, 21)
    slow = 0
    for s in range(5):
        pi = synth.gaussian_pi(30 + s, 400, 20, np.float64)
        rp = metrics.ratios(a, krylov.block_krylov(a, 10, 2, pi).Z, 10, sigma=sig)
        rk = metrics.ratios(a, krylov.block_krylov(a, 10, 2, pi[:, :10]).Z, 10, sigma=sig)
        assert rp["per_vector"] <= 1.001 and rp["spectral"] <= 1.001
        slow += int(rk["per_vector"] > 1.01)
    assert slow >= 4


def test_block_p_rejects_fewer_than_k_columns():
    a, _, _ = _planted(30, 20, 1.0 / np.arange(1, 21), 1)
    with pytest.raises(ValueError):
        krylov.block_krylov(a, 5, 1, synth.gaussian_pi(1, 20, 4, np.float64))


def test_q_capped_when_width_exceeds_dimension():
    a, _, _ = _planted(64, 48, 1.0 / np.arange(1, 49), 5)
    res = krylov.block_krylov(a, 16, 4, synth.gaussian_pi(2, 48, 16))
    assert res.q_eff == 2 and res.Q.shape == (64, 48)
    assert np.allclose(res.sigma, 1.0 / np.arange(1, 17), rtol=1e-11)


def test_simul_iter_converges_to_top_subspace_with_gap():
    sig = 2.0 ** -np.arange(0, 30, dtype=float)
    a, u, v = _planted(80, 30, sig, 13)
    res = krylov.simul_iter(a, 4, 40, synth.gaussian_pi(3, 30, 4))
    assert np.allclose(res.sigma, sig[:4], rtol=1e-12)
    assert metrics.subspace_distance(res.Z, u[:, :4]) < 1e-10


# -------------------------------------------------------------- invariants
def _noisy(n=200, d=120, seed=21):
    sig = np.exp(-np.arange(1, min(n, d) + 1) / 15.0)
    a, _, _ = _planted(n, d, sig, seed)
    a = a + 1e-3 * np.random.default_rng(seed).standard_normal((n, d))
    return a


@pytest.mark.parametrize("method", ["bki", "si"])
def test_orthonormality_span_and_galerkin(method):
    a = _noisy()
    k, q = 5, 4
    pi = synth.gaussian_pi(4, a.shape[1], k)
    res = (krylov.block_krylov if method == "bki" else krylov.simul_iter)(a, k, q, pi)
    w = res.Q.shape[1]
    assert w == (k * (q + 1) if method == "bki" else k)
    assert np.allclose(res.Q.T @ res.Q, np.eye(w), atol=1e-12)
    assert np.allclose(res.Z.T @ res.Z, np.eye(k), atol=1e-12)
    # Z inside span(Q)
    assert np.linalg.norm(res.Z - res.Q @ (res.Q.T @ res.Z)) < 1e-12
    # M is Q^T A A^T Q by definition
    m_def = res.Q.T @ (a @ (a.T @ res.Q))
    assert np.allclose(res.M, m_def, atol=1e-12)
    # Galerkin condition of Rayleigh-Ritz: Q^T (A A^T Z - Z Sigma^2) = 0
    resid = res.Q.T @ (a @ (a.T @ res.Z) - res.Z * res.sigma ** 2)
    assert np.max(np.abs(resid)) < 1e-12 * res.sigma[0] ** 2
    # Ritz values never exceed the true singular values (Sec. 6, used in Thm. 10)
    s = np.linalg.svd(a, compute_uv=False)
    assert np.all(res.sigma <= s[:k] * (1 + 1e-12))
    # Ritz vectors are the ones Lemma 4.1 describes: (Q Ubar_k)(Q Ubar_k)^T A = Q (Q^T A)_k
    qta = res.Q.T @ a
    uu, ss, vvt = np.linalg.svd(qta, full_matrices=False)
    best = (uu[:, :k] * ss[:k]) @ vvt[:k]
    assert np.allclose(res.Z @ (res.Z.T @ a), res.Q @ best, atol=1e-11)
    assert np.allclose(res.sigma, ss[:k], rtol=1e-11)


def test_basis_spans_explicit_krylov_matrix():
    a = _noisy(60, 40, 3)
    k, q = 3, 2
    pi = synth.gaussian_pi(5, 40, k)
    res = krylov.block_krylov(a, k, q, pi)
    kmat = krylov.krylov_matrix(a, k, q, pi)
    # every column of the explicit K lies in span(Q) ...
    rel = np.linalg.norm(kmat - res.Q @ (res.Q.T @ kmat), axis=0) / np.linalg.norm(kmat, axis=0)
    assert np.max(rel) < 1e-10
    # ... and Q spans nothing more than K (same dimension, K full rank here)
    assert np.linalg.matrix_rank(kmat) == res.Q.shape[1]


def test_ritz_values_monotone_in_q():
    a = _noisy(150, 90, 8)
    k = 4
    pi = synth.gaussian_pi(6, 90, k)
    prev = np.zeros(k)
    for q in range(0, 6):
        res = krylov.block_krylov(a, k, q, pi)
        assert np.all(res.sigma >= prev * (1 - 1e-12))
        prev = res.sigma


def test_block_krylov_captures_at_least_simultaneous_iteration():
    # span(K_SI) is inside span(K_BKI), so Lemma 4.1 gives BKI the larger energy for every l
    a = _noisy(150, 90, 9)
    k, q = 6, 3
    pi = synth.gaussian_pi(7, 90, k)
    e_b = metrics.captured_energy(a, krylov.block_krylov(a, k, q, pi).Z)
    e_s = metrics.captured_energy(a, krylov.simul_iter(a, k, q, pi).Z)
    assert np.all(e_b >= e_s * (1 - 1e-12))


# ----------------------------------------------------------- special cases
def test_q0_is_sketch_and_solve():
    a = _noisy(100, 70, 4)
    k = 5
    pi = synth.gaussian_pi(8, 70, k)
    rb = krylov.block_krylov(a, k, 0, pi)
    rs = krylov.simul_iter(a, k, 0, pi)
    q0 = np.linalg.qr(a @ pi.astype(np.float64))[0]
    uu, ss, _ = np.linalg.svd(q0.T @ a, full_matrices=False)
    assert np.allclose(rb.sigma, ss[:k], rtol=1e-12)
    assert np.allclose(rs.sigma, ss[:k], rtol=1e-12)
    assert metrics.subspace_distance(rb.Z, q0 @ uu[:, :k]) < 1e-10


def test_simul_iter_k1_is_power_method():
    a = _noisy(90, 60, 10)
    pi = synth.gaussian_pi(9, 60, 1)
    q = 7
    x = a @ pi[:, 0].astype(np.float64)
    x /= np.linalg.norm(x)
    for _ in range(q):
        x = a @ (a.T @ x)
        x /= np.linalg.norm(x)
    res = krylov.simul_iter(a, 1, q, pi)
    assert abs(abs(res.Z[:, 0] @ x) - 1) < 1e-12
    assert abs(res.sigma[0] - np.linalg.norm(a.T @ x)) < 1e-12


def test_diagonal_matrix_gives_coordinate_vectors():
    a = np.zeros((10, 8))
    vals = [3.0, 7.0, 1.0, 5.0, 2.0, 4.0]
    for i, v in enumerate(vals):
        a[i + 1, i] = v
    res = krylov.block_krylov(a, 2, 2, synth.gaussian_pi(10, 8, 2))   # w = 6 = rank
    assert np.allclose(res.sigma, [7.0, 5.0], rtol=1e-12)
    assert np.allclose(res.Z[:, 0], np.eye(10)[:, 2], atol=1e-12)
    assert np.allclose(res.Z[:, 1], np.eye(10)[:, 4], atol=1e-12)


def test_centred_operator_matches_definition():
    row_ptr, col_idx, vals, d = synth.zipf_idf_csr(n=300, d=120, per_row=7, seed=3)
    mu = synth.column_means(row_ptr, col_idx, vals, 300, d)
    op = krylov.centred_csr_op(row_ptr, col_idx, vals, 300, d, mu)
    dense = np.zeros((300, d))
    for i in range(300):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            dense[i, col_idx[p]] += vals[p]
    dense -= mu.astype(np.float64)[None, :]
    x = np.random.default_rng(0).standard_normal((d, 3))
    y = np.random.default_rng(1).standard_normal((300, 3))
    assert np.allclose(op.mul(x), dense @ x, atol=1e-10)
    assert np.allclose(op.tmul(y), dense.T @ y, atol=1e-10)
    pi = synth.gaussian_pi(3, d, 4)
    r_op = krylov.block_krylov(op, 4, 3, pi)
    r_de = krylov.block_krylov(dense, 4, 3, pi)
    assert np.allclose(r_op.sigma, r_de.sigma, rtol=1e-10)


def test_zipf_rows_are_duplicate_free_and_sorted():
    row_ptr, col_idx, vals, d = synth.zipf_idf_csr(n=500, d=2000, per_row=50, seed=1)
    c = col_idx.reshape(500, 50)
    assert np.all(np.diff(c, axis=1) > 0)
    assert np.all(vals >= 0)


# ----------------------------------------------------- metrics + worked example
def test_worked_example_metrics():
    with open(os.path.join(GOLDEN, "worked_example.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        k = case["k"]
        top = np.full(k + 1, math.sqrt(case["top_sq"]))
        tail = np.full(case["tail_count_per_k"] * k, math.sqrt(case["tail_sq"]))
        s = np.concatenate([top, tail])
        a = np.diag(s)
        rg = np.random.default_rng(k)
        for trial in range(3):
            if trial == 0:   # the oracle's own answer
                z = krylov.block_krylov(a, k, 2, synth.gaussian_pi(k, a.shape[1], k)).Z
            else:            # any orthonormal Z
                z = np.linalg.qr(rg.standard_normal((a.shape[0], k)))[0]
            r = metrics.ratios(a, z, k, sigma=s)
            assert abs(r["spectral"] ** 2 * s[k] ** 2 - case["spectral_sq"]) < 1e-9
            assert r["frobenius"] ** 2 <= case["frobenius_sq_ratio_max"]


def test_metrics_zero_error_for_true_vectors():
    sig = 1.0 / np.arange(1, 31)
    a, u, v = _planted(50, 30, sig, 2)
    r = metrics.ratios(a, u[:, :5], 5, sigma=sig)
    assert abs(r["spectral"] - 1) < 1e-12
    assert abs(r["frobenius"] - 1) < 1e-12
    assert abs(r["per_vector"] - 1) < 1e-12
    # a wrong vector order leaves the subspace (spectral, Frobenius) unchanged
    # but the per-vector error sees it
    r2 = metrics.ratios(a, u[:, [1, 0, 2, 3, 4]], 5, sigma=sig)
    assert abs(r2["spectral"] - 1) < 1e-12 and r2["per_vector"] > 1.5


# ---------------------------------------------------- paper guarantees, C1
def test_guarantees_on_planted_500x300():
    a, sig, u, v = synth.dense_planted_small()
    fails = {"spectral": 0, "frobenius": 0, "per_vector": 0}
    for s in range(5):
        res = krylov.block_krylov(a, 10, 6, synth.gaussian_pi(1 + s, 300, 10))
        r = metrics.ratios(a, res.Z, 10, sigma=sig)
        for key in fails:
            fails[key] += int(r[key] > 1.01)
    assert all(v <= 1 for v in fails.values()), fails


def test_planted_ritz_values_approach_one_over_i():
    a, sig, _, _ = synth.dense_planted_small()
    pi = synth.gaussian_pi(1, 300, 10)
    errs = []
    for q in (1, 3, 6):
        res = krylov.block_krylov(a, 10, q, pi)
        errs.append(np.max(np.abs(res.sigma - sig[:10]) / sig[:10]))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3


# ----------------------------------------------------------------------- RNG
def test_splitmix64_known_answer():
    with open(os.path.join(GOLDEN, "splitmix64.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        assert rng.splitmix64(case["seed"], case["index"]) == int(case["value_hex"], 16)


def test_box_muller_statistics():
    pi = rng.start_block(12345, 5000, 10).astype(np.float64).ravel()
    assert abs(pi.mean()) < 0.02
    assert abs(pi.var() - 1) < 0.03
    from scipy import stats
    assert stats.kstest(pi, "norm").pvalue > 1e-3
    # each pair lies on the circle of radius sqrt(-2 ln u1)
    c, s = rng.gaussian_pair(99, 3)
    x1 = rng.splitmix64(99, 6)
    u1 = ((x1 >> 11) + 1) * 2.0 ** -53
    assert abs(c * c + s * s + 2 * math.log(u1)) < 1e-12


# ------------------------------------------------------------------ gradient
def test_gradient_matches_central_differences():
    rg = np.random.default_rng(1005)
    sig = 1.0 / np.arange(1, 49)
    a, _, _ = _planted(64, 48, sig, 1005)
    a = a + 1e-3 * rg.standard_normal((64, 48))
    t = synth.loss_target(77, 64, 48)
    g = grad.loss_grad(a, 16, t)
    g_fd = grad.central_difference(a, 16, t)
    rel = np.linalg.norm(g - g_fd) / np.linalg.norm(g)
    assert rel < 1e-7, rel


def test_gradient_terms_are_all_needed():
    # each term of the adjoint is visible: dropping the pair sum or the complement
    # term moves the result far outside the finite-difference error
    rg = np.random.default_rng(3)
    a, _, _ = _planted(20, 12, 1.0 / np.arange(1, 13), 3)
    a = a + 1e-3 * rg.standard_normal((20, 12))
    t = synth.loss_target(5, 20, 12)
    k = 4
    _, _, _, ak = grad.truncated(a, k)
    g_full = grad.loss_grad(a, k, t)
    g_fd = grad.central_difference(a, k, t)
    assert np.linalg.norm(g_full - g_fd) / np.linalg.norm(g_fd) < 1e-6
    u, s, v, _ = grad.truncated(a, k)
    gg = 2 * (ak - t)
    comp = (gg @ v[:, :k] - u @ (u.T @ (gg @ v[:, :k]))) @ v[:, :k].T
    assert np.linalg.norm(comp) / np.linalg.norm(g_fd) > 1e-3


# ------------------------------------------------------------- adaptive iteration count
def test_adaptive_stops_once_the_space_covers_the_rank():
    # rank 20, k = 10: two blocks span range(A), so the third adds nothing and the
    # iteration stops there with q = 2; the result is block_krylov's at q = 2
    sig = np.concatenate([1.0 / np.arange(1, 21), np.zeros(20)])
    a, u, v = _planted(60, 40, sig, 13)
    pi = synth.gaussian_pi(4, 40, 10, np.float64)
    res, deltas = krylov.block_krylov_adaptive(a, 10, 8, 1e-10, pi)
    assert res.q_eff == 2 and deltas[-1] < 1e-12 and deltas[0] > 1e-6
    ref = krylov.block_krylov(a, 10, 2, pi)
    assert np.array_equal(res.sigma, ref.sigma)
    assert np.max(np.abs(res.sigma - sig[:10]) / sig[:10]) < 1e-12


def test_adaptive_runs_q_max_when_tol_is_never_met():
    a, _, _, _ = synth.dense_planted_small()
    pi = synth.gaussian_pi(1, 300, 10, np.float64)
    res, deltas = krylov.block_krylov_adaptive(a, 10, 3, 1e-15, pi)
    assert res.q_eff == 3 and len(deltas) == 2 and min(deltas) > 1e-15   # tested after blocks 2 and 3
    ref = krylov.block_krylov(a, 10, 3, pi)
    assert np.array_equal(res.sigma, ref.sigma)


def test_adaptive_changes_are_nonnegative_and_ritz_values_monotone():
    # nested spaces: Ritz values only grow (Courant-Fischer), so every change is an increase
    a, _ = synth.dense_planted_noisy(n=800, d=500, rank=100, seed=6)
    pi = synth.gaussian_pi(2, 500, 8, np.float64)
    op = krylov.dense_op(a)
    prev = None
    for q in range(0, 5):
        s = krylov.block_krylov(a, 8, q, pi).sigma
        if prev is not None:
            assert np.all(s >= prev - 1e-12 * s[0])
        prev = s
    res, deltas = krylov.block_krylov_adaptive(a, 8, 6, 1e-6, pi)
    assert all(d >= 0 for d in deltas) and res.q_eff <= 6


def test_adjoint_from_truncated_triplets_when_they_span_the_range():
    """adjoint_from_triplets with only the leading r' of the triplets: exact (against central
    differences) when A has rank <= r', i.e. when the given triplets span range(A) -- the
    situation of a Krylov space that holds range(A).  With a triplet of the range left out
    it is not (the pin bites)."""
    rng = np.random.default_rng(41)
    n, d, rank, k = 30, 24, 9, 4
    u0 = np.linalg.qr(rng.standard_normal((n, rank)))[0]
    v0 = np.linalg.qr(rng.standard_normal((d, rank)))[0]
    a = (u0 * (1.0 / np.arange(1, rank + 1))) @ v0.T
    t = rng.standard_normal((n, d))
    u, s, v, ak = grad.truncated(a, k)
    g_ak = 2.0 * (ak - t)
    fd = grad.central_difference(a, k, t)
    r = 12   # >= rank
    got = grad.adjoint_from_triplets(u[:, :r], s[:r], v[:, :r], k, np.ones(k), g_ak)
    assert np.linalg.norm(got - fd) / np.linalg.norm(fd) < 1e-6
    short = grad.adjoint_from_triplets(u[:, :rank - 1], s[:rank - 1], v[:, :rank - 1], k, np.ones(k), g_ak)
    assert np.linalg.norm(short - fd) / np.linalg.norm(fd) > 1e-3
