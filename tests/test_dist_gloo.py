"""Multi-process host logic on CPU (gloo, world size 2): instance sharding has one
owner per instance and the timing reductions take the maximum / sum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2409_11382_gb300 import dist as D  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = D.shard(64, rank, world)
        t = 10.0 + rank  # per-rank "timings"
        q.put((rank, mine, D.max_over_ranks(t), D.sum_over_ranks(len(mine))))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_shard_and_reductions_world2():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    owned = sorted(i for _, mine, _, _ in out for i in mine)
    assert owned == list(range(64))                       # every instance exactly once
    assert all(mx == 11.0 for _, _, mx, _ in out)         # max over ranks
    assert all(sm == 64.0 for _, _, _, sm in out)         # sum over ranks


def test_shard_single_process():
    assert D.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert D.shard(5, 1, 2) == [1, 3]
    with pytest.raises(ValueError):
        D.shard(5, 2, 2)
    assert D.max_over_ranks(3.5) == 3.5
