"""The multi-GPU form of bench.py is replicas only (one independent job per
rank, no data-path collective): each rank seeds its own job, the timed region
is bracketed by barriers, and the reported time is the slowest rank's.  The
host side of that is checked here with two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r "measured" 10 (r + 1) ms timed and 20 (r + 1) ms end to end
        ms, e2e = bench.slowest_rank_ms([10.0 * (rank + 1), 20.0 * (rank + 1)], dist, torch.device("cpu"))
        out[rank] = (ms, e2e, bench.replica_seed(1307, rank), bench.whole_job_rate(world, 3, 200, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_report_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        ms, e2e, seed, rate = res[r]
        assert ms == 20.0 and e2e == 40.0  # every rank sees the max over ranks
        assert rate == pytest.approx(2 * 3 * 200 / 0.020)
    assert res[0][2] != res[1][2]  # independent jobs


def test_single_process_needs_no_group():
    import bench
    assert bench.slowest_rank_ms([5.0, 7.0], None, None) == [5.0, 7.0]
    assert bench.whole_job_rate(1, 2, 200, 400.0) == pytest.approx(1000.0)
