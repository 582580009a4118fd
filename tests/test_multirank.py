"""bench.py's multi-GPU path on CPU: two gloo ranks, replicas only (the
method does not shard), the job latency is the slowest replica's."""
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
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {"ms_per_step": 10.0 + 5.0 * rank, "p50_ms": 9.0 + rank, "p99_ms": 12.0 + 7 * rank}
    bench.aggregate_replicas(res, device="cpu")
    out[rank] = (res["value"], res["p50_ms"], res["p99_ms"], res["n_gpus"])
    dist.destroy_process_group()


def test_replica_aggregation_two_gloo_ranks():
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
    assert out[0] == out[1] == (15.0, 10.0, 19.0, 2)
