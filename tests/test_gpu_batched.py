"""GPU parity of the batched entry point: every solve of a batch equals the single solve
of the same matrix with the same start block and the batch's SM budget (bitwise: the same
kernels with the same grids run, only on other streams), and the Ritz values match the FP64 oracle (relative 1e-5, FP32) on the
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
    sms = bk.batch_budget(ams, k, q)
    assert sms > 0
    for i, (a, (z, s, v)) in enumerate(zip(mats, outs)):
        z1, s1, v1 = bk.block_krylov(ams[i], k, q, pi=pis[i], want_v=True, max_sms=sms)
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
    sms = bk.batch_budget([csr, dense, small], 8, 3)
    for seed, m, (z, s) in zip([1, 2, 3], [csr, dense, small], outs):
        z1, s1 = bk.block_krylov(m, 8, 3, seed=seed, max_sms=sms)
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
    sms = bk.batch_budget(ams, k, q)
    for i in (0, 77, 255):
        z1, s1 = bk.block_krylov(ams[i], k, q, seed=i, max_sms=sms)
        assert torch.equal(outs[i][0], z1) and torch.equal(outs[i][1], s1)


def test_autotune_caches_a_budget_and_batches_reuse_it():
    """bks_batched_autotune times the candidate SM budgets, returns the results of the
    fastest, and caches it: a later batched call with max_sms = 0 uses it and equals the
    single calls made with it; an explicit max_sms applies to every matrix of a batch."""
    mats = synth.batched_planted(batch=24, k=16, seed=2005, m_range=(256, 1024), n_range=(128, 512))
    k, q = 16, 4
    ams = [dev(a) for a in mats]
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    before = bk.batch_budget(ams, k, q)
    assert before == max(n_sm // 8, 8)
    outs, best, ms = bk.batched_autotune(ams, k, q, seeds=list(range(24)))
    assert best in (n_sm // 16, n_sm // 8, n_sm // 4, n_sm // 2, n_sm) and ms > 0
    assert bk.batch_budget(ams, k, q) == best
    again = bk.block_krylov_batched(ams, k, q, seeds=list(range(24)))
    for i in (0, 11, 23):
        z1, s1 = bk.block_krylov(ams[i], k, q, seed=i, max_sms=best)
        assert torch.equal(again[i][0], z1) and torch.equal(again[i][1], s1)
        assert torch.equal(outs[i][0], z1) and torch.equal(outs[i][1], s1)
    explicit = bk.block_krylov_batched(ams, k, q, seeds=list(range(24)), max_sms=n_sm)
    z1, s1 = bk.block_krylov(ams[5], k, q, seed=5)
    assert torch.equal(explicit[5][0], z1) and torch.equal(explicit[5][1], s1)


def test_batch_at_the_full_shape_ranges():
    """32 matrices drawn from the batched workload's full ranges (m in [256, 4096], n in
    [128, 2048], sigma_i = 1/i plus 1e-3 noise, k = 16, q = 4): every member equals its single
    call at the batch's SM budget bit for bit, and a sample of three matches the FP64 oracle
    (relative 1e-5 on the Ritz values)."""
    mats = synth.batched_planted(batch=32, k=16, seed=1005)
    k, q = 16, 4
    ams = [dev(a) for a in mats]
    pis = [dev(synth.gaussian_pi(300 + i, a.shape[1], k)) for i, a in enumerate(mats)]
    outs, _, statuses = bk.block_krylov_batched(ams, k, q, pis=pis, stats=True)
    assert all(s in (0, 100) for s in statuses)
    sms = bk.batch_budget(ams, k, q)
    for i in range(32):
        z1, s1 = bk.block_krylov(ams[i], k, q, pi=pis[i], max_sms=sms)
        assert torch.equal(outs[i][0], z1) and torch.equal(outs[i][1], s1), i
    for i in (0, 13, 31):
        ref = krylov.block_krylov(mats[i].astype(np.float64), k, q, pis[i].cpu().numpy())
        sg = outs[i][1].double().cpu().numpy()
        assert np.max(np.abs(sg - ref.sigma) / ref.sigma) <= 1e-5, i
