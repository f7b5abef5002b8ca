"""The N > 1 path of bench.py (independent replicas, no data-path collective)
on CPU: two gloo ranks reduce their per-rank step times and edge counts the way
the GPU run does -- value = edges of all ranks / the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [10.0, 12.5][rank]
        edges = [4e9, 4e9][rank]
        value, step_ms = bench.replica_value(dist, edges, ms, "cpu")
        out[rank] = (value, step_ms, bench.reduce_over_ranks(dist, float(rank + 1), "sum", "cpu"))
    finally:
        dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        value, step_ms, s = res[r]
        assert step_ms == 12.5                              # max over ranks
        assert abs(value - 8e9 / 12.5e-3 / 1e9) < 1e-9      # all ranks' edges / slowest time
        assert s == 3.0


def test_single_process_is_identity():
    import bench
    v, ms = bench.replica_value(None, 2e9, 4.0, "cpu")
    assert ms == 4.0 and abs(v - 500.0) < 1e-9
