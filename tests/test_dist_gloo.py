"""The multi-GPU host path with world_size 2 on CPU (gloo): slowest-rank timing,
block-cyclic shards of tiles and of batch contexts that cover every item exactly
once, and the gather of per-rank output blocks to rank 0."""
import os
import socket

import numpy as np
import pytest

from paper_2505_00448_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    res["max"] = D.max_over_ranks(10.0 + 5.0 * rank, dist)
    res["sum"] = D.sum_over_ranks(rank + 1, dist)
    # a rank's share of a 1,000-variable triangle of 128x128 tiles and of 256 contexts
    tiles = D.shard_triangle(1000, 128, world, rank, block=8)
    ctxs = D.shard_blocks(256, world, rank, block=1)
    # each rank "computes" its output blocks (a stand-in value per tile) and
    # rank 0 gathers them
    blocks = {t: (t[0] * 1000 + t[1]) * 1.0 for t in tiles}
    res["gathered"] = D.gather_to_root({"tiles": tiles, "ctxs": ctxs, "blocks": blocks}, dist)
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(outdir, f"r{rank}.npy"), np.array([res], dtype=object), allow_pickle=True)


def test_world2_gloo(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "r0.npy", allow_pickle=True)[0]
    r1 = np.load(tmp_path / "r1.npy", allow_pickle=True)[0]
    assert r0["max"] == r1["max"] == 15.0
    assert r0["sum"] == r1["sum"] == 3.0
    assert r1["gathered"] is None
    g = r0["gathered"]
    assert len(g) == 2
    all_tiles = D.triangle_tiles(1000, 128)
    got = g[0]["tiles"] + g[1]["tiles"]
    assert sorted(got) == sorted(all_tiles) and len(set(got)) == len(all_tiles)
    assert sorted(g[0]["ctxs"] + g[1]["ctxs"]) == list(range(256))
    merged = {**g[0]["blocks"], **g[1]["blocks"]}
    assert all(merged[t] == (t[0] * 1000 + t[1]) * 1.0 for t in all_tiles)


def test_shards_cover_once_any_world():
    for world in (1, 2, 3, 4, 8):
        for n, block in ((0, 1), (7, 1), (256, 1), (1000, 8), (37, 5)):
            parts = [D.shard_blocks(n, world, r, block) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert sorted(flat) == list(range(n)) and len(flat) == n
    with pytest.raises(ValueError):
        D.shard_blocks(10, 2, 2)
    assert D.weak_scaling_value(100, 2.0, 4) == 200.0
