"""Host logic of the N > 1 paths on CPU ranks (gloo, world size 2): the
size-balanced split of independent scenes over GPUs, the max/sum of the
per-rank timing results that bench.py prints, and bench.py's batched leg
end to end with stub scene runners (no GPU)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _StubScene:
    def __init__(self, i, precision):
        self.i, self.nv, self.precision = i, 4, precision

    def bbox_diag(self):
        return 2.0


class _StubScenes:
    """scene sizes from the real generator's draws; stub meshes"""

    @staticmethod
    def batch_scene_size(i):
        from paper_2512_12151_b300 import scenes
        return scenes.batch_scene_size(i)

    @staticmethod
    def batch_scene(i, precision=1):
        return _StubScene(i, precision)


class _StubServing:
    """the real split; batch and sequential runners that return fixed
    timings per scene and end states that differ by 1e-6 per precision"""

    def __init__(self, rank):
        self.rank = rank

    @staticmethod
    def shard(sizes, world):
        from paper_2512_12151_b300 import serving
        return serving.shard(sizes, world)

    def run_batched(self, mix, n_steps, n_workers):
        return {"steps": n_steps * len(mix), "seconds": 1.0 + self.rank}, [((s.i, 1), None) for s in mix]

    def run_sequential(self, mix, n_steps):
        return {"steps": n_steps * len(mix), "seconds": 10.0 + self.rank}, [((s.i, 0), None) for s in mix]

    @staticmethod
    def destroy(hs):
        pass


class _StubB:
    @staticmethod
    def bf_get_state(h, nv):
        i, mixed = h
        return np.full((nv, 3), float(i)) + 1e-6 * mixed, None


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
    batched, plain = bench.batched_leg(world, rank, 64, 4, _StubScenes, _StubServing(rank), _StubB)
    out.put((rank, parts, tmax, tsum, sizes, batched, plain))
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
    res.sort(key=lambda r: r[0])
    sizes = res[0][4]
    parts = res[0][1]
    assert res[1][1] == parts  # every rank sees the same split
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(sizes)))  # each scene on exactly one rank
    loads = [sum(sizes[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(sizes)  # greedy balance bound
    assert all(r[2] == 2.0 for r in res)  # max over ranks
    assert all(r[3] == float(sum(sizes)) for r in res)  # sum over ranks
    # the batched leg: the whole list is advanced once over both ranks, the
    # time is the slowest rank's, the deviation the largest over the ranks
    for r in res:
        batched, plain = r[5], r[6]
        assert batched["scenes_per_rank"] == [len(p) for p in parts]
        assert batched["steps_per_s"] == 10 * 64 / 2.0
        assert plain["steps_per_s"] == 10 * 64 / 11.0
        assert abs(batched["max_deviation_from_fp64"] - 1e-6 / 2.0) < 1e-15
