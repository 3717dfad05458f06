"""The N > 1 bench path on CPU: two gloo ranks, each with its own scene seed,
no collective on the data path; the step time is the max over ranks."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_2604_26799_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        assert (ws, r, local) == (world, rank, rank)
        # each rank owns a different scene: no data exchange between ranks
        attrs, _ = synth.make_scene(1000, seed=synth.SCENE.seed + r)
        bench.barrier(ws)
        t = bench.reduce_max(float(rank + 1) * 10.0, ws)
        out[rank] = (t, float(attrs[0, 0]))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_timing_and_distinct_scenes():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    assert res[0][1] != res[1][1]
