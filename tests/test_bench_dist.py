"""The multi-rank logic of bench.py on CPU: two gloo ranks (127.0.0.1) each
time their own shard; the reported time is the slowest rank's, the value
counts every rank's paths, and the shards draw different inputs."""
import os
import socket

import numpy as np
import pytest

import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ws, r, local = bench._dist()
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        seed = bench.shard_seed(r)
        y, _ = W.random_points(seed, 64, 4)
        q.put((r, ws, local, slowest, seed, y[0, 0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[3] == 15.0 for o in out)          # both ranks see the slowest rank's time
    assert out[0][4] != out[1][4]                   # distinct shard seeds
    assert out[0][5] != out[1][5]                   # hence distinct inputs


def test_single_process_and_rate():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5   # no process group: the value itself
    assert bench.whole_job_rate(2, 65536, 0.5) == pytest.approx(262144.0)
    assert bench.whole_job_rate(1, 65536, 0.5) == pytest.approx(131072.0)
