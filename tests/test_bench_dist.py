"""The multi-GPU path of bench.py is replicas only: each rank acquires its own
recordings, the job time is the slowest rank's (max over ranks) and the
whole-job value sums every rank's cells.  Checked with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [10.0, 14.0, 12.0][rank]
    mx = bench.reduce_max_over_ranks(local_ms, torch.device("cpu"))
    dist.barrier()
    q.put((rank, mx, bench.job_value(1000.0, 5, world, mx)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_aggregation_with_gloo(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([10.0, 14.0, 12.0][:world])
    for rank, mx, val in out:
        assert mx == slowest
        assert val == pytest.approx(world * 1000.0 * 5 / (slowest * 1e-3))


def test_single_process_needs_no_group():
    import bench
    assert bench.reduce_max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert bench.job_value(10.0, 2, 1, 4.0) == pytest.approx(5000.0)
