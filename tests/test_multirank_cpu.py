"""The multi-GPU host logic of the benchmark on CPU: two gloo ranks.  Images
are independent units (replicas), so the only cross-rank step is the max of the
per-rank timings; the whole-job value counts every rank's units over the
slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as td

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [120.0, 150.0][rank]  # rank 1 is the slower one
    slowest = bench.rank_max(local_ms, device="cpu")
    value = bench.whole_job_value(2_073_600 * 10 * 5, world, slowest)
    q.put((rank, slowest, value))
    td.barrier()
    td.destroy_process_group()


def test_two_ranks_max_timing_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, slowest, value in res:
        assert slowest == 150.0
        assert value == pytest.approx(2 * 2_073_600 * 10 * 5 / 0.150 / 1e6)


def test_single_process_identity():
    import bench

    assert bench.rank_max(3.5, device="cpu") == 3.5
    assert bench.whole_job_value(1e6, 1, 1000.0) == pytest.approx(1.0)
