"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each timing
its own independent problem; the job reports the slowest rank's time and all
ranks' units over it (weak scaling, no data-path collective), and the ranks'
nodal fields differ."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, rate = bench.whole_job_rate(10.0 * (rank + 1), 100, 5, dist)
    seeds = [bench.rank_field_seed(rank, s) for s in range(4)]
    q.put((rank, ms, rate, seeds))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_slowest_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    for rank, ms, rate, _ in out:
        assert ms == 20.0                          # the slower rank's time on every rank
        assert rate == pytest.approx(2 * 100 * 5 / 0.020)
    assert not set(out[0][3]) & set(out[1][3])     # independent fields per rank


def test_single_process_rate():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.whole_job_rate(4.0, 1000, 10, None)
    assert ms == 4.0 and rate == pytest.approx(1000 * 10 / 0.004)
