"""Replica timing across ranks (bench.py under torchrun): max time, summed work.

Runs two gloo processes on the CPU; each rank reports its own time and units."""
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
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_1207_2223_gb300 import replicas
    r, size = replicas.init("gloo")
    assert (r, size) == (rank, world)
    replicas.barrier()
    t, u = replicas.combine(1.5 + rank, 5 + 2 * rank)
    out.put((rank, t, u))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_combine_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u in res:
        assert t == 2.5           # max over ranks
        assert u == 12.0          # 5 + 7 units


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_1207_2223_gb300 import replicas
    assert replicas.world() == (0, 1, 0)
    assert replicas.combine(3.0, 4) == (3.0, 4.0)
