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


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    import bench
    from paper_2605_16564_gb300 import fields
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        for name in ("layered3d_quarter", "voronoi2d"):
            W = bench.WORKLOADS[name]
            b, e = bench.shard_ranges(bench.shard_costs(W), world)[rank]
            h = fields.cell_size(W["shape"])
            pts = fields.cell_centred_points(W["eval_counts"], [n * h for n in W["shape"]])
            own = bench.owner_index(W, pts)
            mine = int(((own >= b) & (own < e)).sum())
            cost = float(bench.shard_costs(W)[b:e].sum())
            ranges = [None] * world
            dist.all_gather_object(ranges, (b, e, mine, cost))
            out[name] = ranges
        # the one collective of a sharded field: this rank's error sums added up
        s = torch.tensor([rank + 1.0] * 6 + [10.0 * rank + 3.0, 0.0], dtype=torch.float64)
        tot = bench.combine_error_sums(s, world)
        q.put((rank, out, tot.tolist()))
    finally:
        dist.destroy_process_group()


def test_one_field_sharded_over_two_gloo_ranks():
    # section 8(e): contiguous blocks of subdomains balanced by N_i M^2, every
    # subdomain and every target point on exactly one rank, the error sums
    # added over the ranks (maximum for the max-norm entry)
    import numpy as np
    import torch.multiprocessing as mp
    import bench
    from paper_2605_16564_gb300 import fields
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for name in ("layered3d_quarter", "voronoi2d"):
        W = bench.WORKLOADS[name]
        S = int(np.prod(W["n_sub"]))
        ranges = res[0][1][name]
        assert ranges == res[1][1][name]  # every rank computed the same plan
        assert ranges[0][0] == 0 and ranges[0][1] == ranges[1][0] and ranges[1][1] == S
        n_pts = int(np.prod(W["eval_counts"]))
        assert ranges[0][2] + ranges[1][2] == n_pts
        costs = [r[3] for r in ranges]
        assert max(costs) <= 1.05 * sum(costs) / 2
    for _, _, tot in res:
        assert tot[:6] == [3.0] * 6 and tot[6] == 13.0
