"""Host logic of the N > 1 paths on CPU ranks (gloo, world size 2): the
size-balanced split of independent scenes over GPUs and the max/sum of the
per-rank timing results that bench.py prints."""
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
    from paper_2512_12151_b300 import scenes, serving
    sizes = [scenes.batch_scene(i).nt for i in range(64)]
    mine = serving.shard(sizes, world)[rank]
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    tmax = bench.allmax(world, 1.0 + rank)
    tsum = bench.allsum(world, float(sum(sizes[i] for i in mine)))
    out.put((rank, parts, tmax, tsum, sizes))
    dist.destroy_process_group()


def test_shard_and_reductions_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    sizes = res[0][4]
    parts = res[0][1]
    assert res[1][1] == parts  # every rank sees the same split
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(sizes)))  # each scene on exactly one rank
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)  # greedy balance bound
    assert all(r[2] == 2.0 for r in res)  # max over ranks
    assert all(r[3] == float(sum(sizes)) for r in res)  # sum over ranks
