"""The multi-rank timing reduction of bench.py (replicas; max over ranks) on
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    bench.dist_init("gloo")
    r, lr, w = bench.dist_env()
    bench.dist_barrier(w)
    out[rank] = bench.dist_max(1.5 + 2.0 * rank, w)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert dict(out) == {0: 3.5, 1: 3.5}


def test_single_rank_is_identity():
    import bench
    assert bench.dist_max(2.25, 1) == 2.25
