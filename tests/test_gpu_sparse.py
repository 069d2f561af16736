"""GPU parity of the sparse path (CSR A, implicit centring A - 1 mu^T) against the FP64
oracle, through the C-ABI.

Tolerances: the CSR transpose is integer/copy work and must match scipy bit for bit;
products accumulate each row segment in FP32 and segments in FP64, so
|Y - Y_ref| <= 4 sqrt(L) eps (|A||X|) with L the longest row (plus the centring term,
which is formed in FP64); Ritz values relative 1e-5; error ratios within 1e-3."""
import numpy as np
import pytest

import synth
from oracle import krylov, metrics

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
sp = pytest.importorskip("scipy.sparse")
bk = pytest.importorskip("paper_1504_05477_gb300")

EPS32 = 2.0 ** -24


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def make(n, d, per_row, seed, empty_rows=()):
    row_ptr, col_idx, vals, d = synth.zipf_idf_csr(n=n, d=d, per_row=per_row, seed=seed)
    if empty_rows:
        a = sp.csr_matrix((vals, col_idx, row_ptr), shape=(n, d)).tolil()
        for r in empty_rows:
            a.rows[r] = []
            a.data[r] = []
        a = a.tocsr()
        a.sort_indices()
        row_ptr, col_idx, vals = a.indptr.astype(np.int64), a.indices.astype(np.int32), a.data.astype(np.float32)
    mu = synth.column_means(row_ptr, col_idx, vals, n, d)
    return row_ptr, col_idx, vals, d, mu


def gpu_csr(row_ptr, col_idx, vals, n, d, mu=None, transpose=True):
    return bk.CsrMatrix(dev(row_ptr), dev(col_idx), dev(vals), (n, d),
                        col_mean=dev(mu) if mu is not None else None, transpose=transpose)


def test_csr_transpose_matches_scipy_bitwise():
    n, d = 5000, 3000
    row_ptr, col_idx, vals, d, _ = make(n, d, 40, 3, empty_rows=(7, 100, 4999))
    a = gpu_csr(row_ptr, col_idx, vals, n, d)
    t_rp, t_ci, t_cv = (host(x) for x in a.t)
    ref = sp.csr_matrix((vals, col_idx, row_ptr), shape=(n, d)).T.tocsr()
    ref.sort_indices()
    assert np.array_equal(t_rp, ref.indptr.astype(np.int64))
    assert np.array_equal(t_ci[:ref.nnz], ref.indices.astype(np.int32))
    assert np.array_equal(t_cv[:ref.nnz].view(np.uint32), ref.data.astype(np.float32).view(np.uint32))


@pytest.mark.parametrize("centred", [False, True])
@pytest.mark.parametrize("trans", [False, True])
def test_sparse_products(centred, trans):
    n, d, c = 20000, 6000, 20
    row_ptr, col_idx, vals, d, mu = make(n, d, 50, 5, empty_rows=(0, 19999))
    a = gpu_csr(row_ptr, col_idx, vals, n, d, mu if centred else None)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((n if trans else d, c)).astype(np.float32)
    y = host(bk.matmul(a, dev(x), trans=trans)).astype(np.float64)
    y2 = host(bk.matmul(a, dev(x), trans=trans)).astype(np.float64)
    assert np.array_equal(y, y2)   # deterministic
    s = sp.csr_matrix((vals.astype(np.float64), col_idx, row_ptr), shape=(n, d))
    m = s.T if trans else s
    x64 = x.astype(np.float64)
    ref = m @ x64
    absd = abs(m) @ np.abs(x64)
    corr = np.zeros_like(ref)
    if centred:
        mu64 = mu.astype(np.float64)
        if trans:
            corr = np.outer(mu64, x64.sum(axis=0))
        else:
            corr = np.outer(np.ones(n), mu64 @ x64)
        ref = ref - corr
    # element-wise: FP32 accumulation of a row's lmax products, the correction (summed in
    # FP64 on the device) rounded once to FP32 and subtracted, the result rounded once
    lmax = np.max(np.diff(m.tocsr().indptr))
    bound = 4 * np.sqrt(lmax) * EPS32 * absd + 2 * EPS32 * np.abs(corr) + 2 * EPS32 * np.abs(ref) + 1e-38
    assert np.all(np.abs(y - ref) <= bound), float(np.max(np.abs(y - ref) / bound))


@pytest.mark.parametrize("method", ["bki", "si"])
def test_sparse_centred_small_parity(method):
    n, d, k, q = 3000, 1500, 20, 10
    row_ptr, col_idx, vals, d, mu = make(n, d, 30, 9)
    a = gpu_csr(row_ptr, col_idx, vals, n, d, mu)
    pi = synth.gaussian_pi(3, d, k)
    fn = bk.block_krylov if method == "bki" else bk.simul_iter
    z, s = fn(a, k, q, pi=dev(pi))
    z, s = host(z).astype(np.float64), host(s).astype(np.float64)
    op = krylov.centred_csr_op(row_ptr, col_idx, vals, n, d, mu)
    ref = (krylov.block_krylov if method == "bki" else krylov.simul_iter)(op, k, q, pi)
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= 1e-5
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 1e-5, np.max(np.abs(z.T @ z - np.eye(k)))
    dense = op.dense()
    sig = metrics.true_singular_values(dense)
    r_gpu = metrics.ratios(dense, z, k, sigma=sig)
    r_ora = metrics.ratios(dense, ref.Z, k, sigma=sig)
    for key in r_gpu:
        assert abs(r_gpu[key] - r_ora[key]) <= 1e-3, key
    if method == "bki":   # eps = 0.05 guarantees of eqs. (1)-(3)
        assert r_gpu["spectral"] <= 1.05 and r_gpu["frobenius"] <= 1.05 and r_gpu["per_vector"] <= 1.05


def test_sparse_centred_full_size_parity():
    """The 200000 x 60000 term-document workload (1e7 non-zeros, k = 20, q = 10), centred."""
    n, d, k, q = 200000, 60000, 20, 10
    row_ptr, col_idx, vals, d, mu = make(n, d, 50, 1003)
    a = gpu_csr(row_ptr, col_idx, vals, n, d, mu)
    pi = synth.gaussian_pi(3, d, k)
    z, s = bk.block_krylov(a, k, q, pi=dev(pi))
    s = host(s).astype(np.float64)
    op = krylov.centred_csr_op(row_ptr, col_idx, vals, n, d, mu)
    ref = krylov.block_krylov(op, k, q, pi)
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= 1e-5
    zz = host(z).astype(np.float64)
    assert np.max(np.abs(zz.T @ zz - np.eye(k))) < 1e-5, np.max(np.abs(zz.T @ zz - np.eye(k)))
    # per-vector captured variance agrees with the oracle's (Z^T A_c through the operator)
    cap_g = np.sum(op.tmul(zz) ** 2, axis=0)
    cap_o = np.sum(op.tmul(ref.Z) ** 2, axis=0)
    assert np.max(np.abs(cap_g - cap_o) / cap_o) <= 2e-5


def test_sparse_without_transpose_matches_with():
    n, d = 8000, 2000
    row_ptr, col_idx, vals, d, mu = make(n, d, 30, 11)
    a1 = gpu_csr(row_ptr, col_idx, vals, n, d, mu, transpose=True)
    a2 = gpu_csr(row_ptr, col_idx, vals, n, d, mu, transpose=False)
    pi = dev(synth.gaussian_pi(4, d, 16))
    _, s1 = bk.block_krylov(a1, 16, 4, pi=pi)
    _, s2 = bk.block_krylov(a2, 16, 4, pi=pi)
    assert np.array_equal(host(s1), host(s2))


def _bad_structures():
    """Small CSR arrays (6 x 5) with one structural defect each."""
    rp = np.array([0, 2, 3, 3, 5, 6, 8], np.int64)
    ci = np.array([0, 3, 1, 2, 4, 0, 1, 4], np.int32)
    out = {}
    dup = ci.copy(); dup[1] = 0                       # repeated column in row 0
    out["duplicate"] = (rp, dup)
    oob = ci.copy(); oob[4] = 5                       # column index == d
    out["column_range"] = (rp, oob)
    neg = ci.copy(); neg[2] = -1
    out["negative_column"] = (rp, neg)
    uns = ci.copy(); uns[3], uns[4] = 4, 2            # row 3 unsorted
    out["unsorted"] = (rp, uns)
    short = rp.copy(); short[-1] = 7                  # row_ptr[n] != nnz
    out["row_ptr_end"] = (short, ci)
    dec = rp.copy(); dec[3] = 2                       # decreasing offsets
    out["row_ptr_order"] = (dec, ci)
    return out


@pytest.mark.parametrize("defect", sorted(_bad_structures()))
def test_sparse_invalid_structure_is_rejected(defect):
    rp, ci = _bad_structures()[defect]
    vals = np.arange(1, ci.size + 1, dtype=np.float32)
    with pytest.raises(bk.BksError) as err:
        gpu_csr(rp, ci, vals, 6, 5)                   # checked by bks_csr_transpose
    assert err.value.status == 1
    a = gpu_csr(rp, ci, vals, 6, 5, transpose=False)  # checked inside the product call
    with pytest.raises(bk.BksError) as err:
        bk.matmul(a, dev(np.ones((5, 3), np.float32)))
    assert err.value.status == 1
    # the context stays usable
    good = gpu_csr(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32),
                   np.array([2.0, 3.0], np.float32), 2, 2)
    y = host(bk.matmul(good, dev(np.eye(2, dtype=np.float32))))
    assert np.array_equal(y, np.array([[0, 2], [3, 0]], np.float32))


@pytest.mark.parametrize("method", ["bki", "si"])
def test_graph_adjacency_centred_parity(method):
    """Square power-law adjacency (the graph workload's shape class), column-centred as
    the paper's principal components, k = 10, q = 6, against the oracle."""
    n, k, q = 6000, 10, 6
    row_ptr, col_idx, vals, n = synth.powerlaw_graph_csr(n=n, seed=8)
    mu = synth.column_means(row_ptr, col_idx, vals, n, n)
    a = gpu_csr(row_ptr, col_idx, vals, n, n, mu)
    pi = synth.gaussian_pi(4, n, k)
    fn = bk.block_krylov if method == "bki" else bk.simul_iter
    z, s = fn(a, k, q, pi=dev(pi))
    z, s = host(z).astype(np.float64), host(s).astype(np.float64)
    op = krylov.centred_csr_op(row_ptr, col_idx, vals, n, n, mu)
    ref = (krylov.block_krylov if method == "bki" else krylov.simul_iter)(op, k, q, pi)
    assert np.max(np.abs(s - ref.sigma) / ref.sigma) <= 1e-5
    assert np.max(np.abs(z.T @ z - np.eye(k))) < 1e-5, np.max(np.abs(z.T @ z - np.eye(k)))
