"""The N>1 path of bench.py runs independent replicas (the product does not shard here):
the job time is the slowest rank's and the value sums all ranks' work.  Checked with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.aggregate_ranks(100.0 + 50.0 * rank, 2e12, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = out[r]
        assert ms == pytest.approx(150.0)                    # slowest rank
        assert value == pytest.approx(2 * 2e12 / 0.150 / 1e9)  # both ranks' flops over it


def test_single_process_aggregation():
    import bench
    ms, value = bench.aggregate_ranks(200.0, 4e12)
    assert ms == 200.0 and value == pytest.approx(20000.0)
