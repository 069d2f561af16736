"""GPU parity of the batched entry point: every solve of a batch equals the single solve
of the same matrix with the same start block (bitwise: the same kernels run, only on
other streams), and the Ritz values match the FP64 oracle (relative 1e-5, FP32) on the
batched workload's shapes (uneven m ~ U[256, 4096], n ~ U[128, 2048], sigma_i = 1/i plus
1e-3 N(0,1) noise, k = 16, q = 4)."""
import numpy as np
import pytest

import synth
from oracle import krylov

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
bk = pytest.importorskip("paper_1504_05477_gb300")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_batch_equals_single_solves_and_oracle():
    mats = synth.batched_planted(batch=12, k=16, seed=1005, m_range=(256, 1024), n_range=(128, 512))
    k, q = 16, 4
    pis = [dev(synth.gaussian_pi(100 + i, a.shape[1], k)) for i, a in enumerate(mats)]
    ams = [dev(a) for a in mats]
    outs, st, statuses = bk.block_krylov_batched(ams, k, q, pis=pis, want_v=True, stats=True)
    assert all(s in (0, 100) for s in statuses)
    assert st["product_launches"] > 0
    for i, (a, (z, s, v)) in enumerate(zip(mats, outs)):
        z1, s1, v1 = bk.block_krylov(ams[i], k, q, pi=pis[i], want_v=True)
        assert torch.equal(z, z1) and torch.equal(s, s1) and torch.equal(v, v1)
        if i < 4:
            ref = krylov.block_krylov(a.astype(np.float64), k, q, pis[i].cpu().numpy())
            sg = s.double().cpu().numpy()
            assert np.max(np.abs(sg - ref.sigma) / ref.sigma) <= 1e-5


def test_batch_mixes_dense_and_sparse_and_reports_per_matrix_status():
    rp, ci, cv, d = synth.zipf_idf_csr(n=3000, d=1000, per_row=20, seed=7)
    csr = bk.CsrMatrix(dev(rp), dev(ci), dev(cv), (3000, d))
    dense = dev(synth.batched_planted(batch=1, k=8, seed=3, m_range=(500, 500), n_range=(300, 300))[0])
    small = dev(np.random.default_rng(1).standard_normal((40, 20)).astype(np.float32))   # q capped
    outs, _, statuses = bk.block_krylov_batched([csr, dense, small], 8, 3, seeds=[1, 2, 3], stats=True)
    assert statuses == [0, 0, 100]
    for seed, m, (z, s) in zip([1, 2, 3], [csr, dense, small], outs):
        z1, s1 = bk.block_krylov(m, 8, 3, seed=seed)
        assert torch.equal(z, z1) and torch.equal(s, s1)
        zz = z.double().cpu().numpy()
        assert np.max(np.abs(zz.T @ zz - np.eye(8))) < 1e-4
        assert torch.all(s[:-1] >= s[1:])


def test_batch_of_256():
    """256 matrices in one call (shapes scaled down from the batched workload so that the
    host generator stays quick; the full-size batch is timed, not tested)."""
    mats = synth.batched_planted(batch=256, k=16, seed=1005, m_range=(256, 1024), n_range=(128, 512))
    k, q = 16, 4
    ams = [dev(a) for a in mats]
    outs, st, statuses = bk.block_krylov_batched(ams, k, q, seeds=list(range(256)), stats=True)
    assert all(s in (0, 100) for s in statuses)
    for i in (0, 77, 255):
        z1, s1 = bk.block_krylov(ams[i], k, q, seed=i)
        assert torch.equal(outs[i][0], z1) and torch.equal(outs[i][1], s1)
