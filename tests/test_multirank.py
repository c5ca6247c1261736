"""The multi-GPU bench logic on CPU ranks (gloo, world size 2): every rank
fits its own field (distinct seeds, no exchange on the data path) and the
step time reported is the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, ws = bench._dist()
        t = bench.max_over_ranks(1.0 + 2.5 * rank, ws)
        bench.barrier(ws)
        seed = bench.shard_seed(5, r)
        q.put((r, ws, t, seed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_step_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _, _ in res] == [0, 1]
    assert all(ws == 2 for _, ws, _, _ in res)
    assert all(t == 3.5 for _, _, t, _ in res)           # max over ranks
    assert res[0][3] != res[1][3]                        # each rank its own field


def test_owner_counts_cover_every_target_point():
    import numpy as np
    import bench
    from paper_2605_16564_gb300 import fields
    for name in ("layered3d_quarter", "voronoi2d", "disc2d"):
        W = bench.WORKLOADS[name]
        h = fields.cell_size(W["shape"])
        pts = fields.cell_centred_points(W["eval_counts"], [n * h for n in W["shape"]])
        c = bench.owner_counts(W, pts)
        assert c.sum() == len(pts) and len(c) == int(np.prod(W["n_sub"]))
