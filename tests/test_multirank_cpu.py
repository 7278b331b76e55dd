"""The N > 1 path of bench.py on CPU: independent replicas, one per rank,
whose whole-job throughput divides the units of all ranks by the slowest
rank's time (max over ranks through torch.distributed, here gloo with
world size 2 on 127.0.0.1)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def mx(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t[0])

    local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
    value, t = bench.aggregate(local_ms, 1e9, world, mx)
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        value, t = res[r]
        assert t == 15.0
        assert abs(value - 2e9 / 15e-3) < 1e-3 * value


def test_single_rank_aggregate():
    import bench
    v, t = bench.aggregate(20.0, 1e9, 1, None)
    assert t == 20.0 and abs(v - 5e10) < 1
