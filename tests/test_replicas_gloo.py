"""Multi-rank host logic on CPU: two gloo processes (no GPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

from paper_2111_14239_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = replicas.world()
    seeds = replicas.image_seeds(2000, 16, r)
    mine = float(10 + 5 * r)          # pretend rank r took 10 + 5r seconds
    slowest = replicas.max_over_ranks(mine)
    dist.barrier()
    q.put((r, w, seeds, slowest, list(replicas.shard(10, r, w))))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, s0, m0, sh0), (r1, w1, s1, m1, sh1) = out
    assert (r0, r1, w0, w1) == (0, 1, 2, 2)
    assert s0 == list(range(2000, 2016)) and s1 == list(range(2016, 2032))   # disjoint images
    assert m0 == m1 == 15.0                                                   # max over ranks
    assert sh0 + sh1 == list(range(10))
    assert replicas.job_throughput(16, 2, 15.0) == pytest.approx(32 / 15.0)


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.world() == (0, 1, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert [len(replicas.shard(10, r, 3)) for r in range(3)] == [4, 3, 3]
