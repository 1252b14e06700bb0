"""The multi-GPU run is N independent replicas; the only collective is the
whole-job total (slowest rank's time, summed particle-steps).  Checked here with
two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, ps = bench.replica_totals(torch, 10.0 + 5.0 * rank, 1000 * (rank + 1), world, "cpu")
        out[rank] = (ms, ps)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_slowest_time_and_summed_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (15.0, 3000.0) and out[1] == (15.0, 3000.0)


def test_one_replica_needs_no_process_group():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(torch, 7.5, 42, 1, "cpu") == (7.5, 42.0)
