"""Multi-process path of the benchmark on CPU: two gloo ranks, each with its own timing,
agree on the slowest time and on the whole-job throughput."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1501_04552_gb300 import replicas
    local_seconds = 1.0 + rank          # rank 1 is the slow one
    slowest = replicas.max_over_ranks(local_seconds)
    out[rank] = (slowest, replicas.throughput(50, world, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_and_throughput():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
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
    assert out[0] == out[1] == (2.0, 50.0)


def test_single_process_is_identity():
    from paper_1501_04552_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.throughput(10, 1, 2.0) == 5.0
