"""Multi-rank bench aggregation on CPU (gloo, world size 2): the job's time is the
maximum over ranks and its work the sum, so `value` is whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [10.0, 20.0] if rank == 0 else [15.0, 25.0]      # ms per step on this rank
    work = 1e9 if rank == 0 else 3e9                          # J.v DOFs on this rank
    total_ms, gdofs = bench.aggregate(times, work, world, rank)
    out[rank] = (total_ms, gdofs)
    dist.destroy_process_group()


def test_aggregate_max_time_sum_work():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        total_ms, gdofs = out[r]
        assert total_ms == pytest.approx(40.0)                # max(30, 40)
        assert gdofs == pytest.approx(4e9 / 0.040 / 1e9)      # (1e9 + 3e9) DOF / 40 ms
