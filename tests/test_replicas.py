"""The multi-GPU path runs independent replicas, one per rank: every rank
times its own copy of the workload and the job's rate is all ranks' units
over the slowest rank's time (bench.replica_rate).  Checked here with two
gloo ranks on the CPU, the slower rank on either side."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, seconds, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        value, slowest = bench.replica_rate(1000.0, seconds[rank], world, dist, torch.device("cpu"))
        out.put((rank, value, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("seconds", [(0.5, 2.0), (3.0, 1.0)])
def test_replica_rate_takes_the_slowest_rank(seconds):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, seconds, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slow = max(seconds)
    for rank, value, slowest in res:
        assert slowest == slow
        assert value == pytest.approx(2 * 1000.0 / slow, rel=1e-15)


def test_replica_rate_single_rank():
    import bench
    assert bench.replica_rate(300.0, 1.5, 1) == (200.0, 1.5)
