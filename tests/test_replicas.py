"""The multi-GPU form is N independent replicas (the build of one graph does
not shard without an exchange step).  The only cross-rank step is the
benchmark's timing: every rank's units over the slowest rank's time.  This
runs it as two gloo ranks on the CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, ms = bench.job_throughput(100.0 * (rank + 1), 2.4e9, world, dist, "cpu")
        out.put((rank, value, ms))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_is_all_units_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms in got:
        assert ms == pytest.approx(200.0)              # the slower rank's time
        assert value == pytest.approx(2 * 2.4e9 / 0.2)  # both ranks' edges over it


def test_single_process_needs_no_collective():
    import bench
    value, ms = bench.job_throughput(80.0, 2.4e9, 1)
    assert ms == 80.0 and value == pytest.approx(3e10)
