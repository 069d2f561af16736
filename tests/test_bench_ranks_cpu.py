"""The multi-rank logic of bench.py on CPU: two gloo ranks, one replica each."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r measured 10 + 5 r ms for its step; the job time is the slowest rank's
    t = bench.job_time(10.0 + 5.0 * rank, world)
    out[rank] = (t, bench.per_solve(t, world, 1), bench.per_solve(t, world, 256))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_max_over_ranks_and_value_counts_all_ranks():
    world, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        t, v1, v256 = out[r]
        assert t == 15.0                  # max(10, 15)
        assert v1 == pytest.approx(7.5)   # 2 solves in 15 ms
        assert v256 == pytest.approx(15.0 / 512)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_time(12.5, 1) == 12.5
    assert bench.per_solve(12.5, 1, 1) == 12.5
