"""The multi-GPU split with world_size 2 on CPU (gloo): each rank computes,
with the FP64 oracle, the output entries its part owns under the library's
split rule (napg_run_part: output rows in blocks of 256 dealt back and forth;
symmetric calls own pair (i, j) by row min(i, j)); rank 0 gathers the blocks,
stitches them and compares with the oracle's unsplit matrices. Also: the
slowest-rank timing, the split throughput, the block-cyclic context shards and
the ownership rule's coverage and balance for other world sizes."""
import os
import socket

import numpy as np
import pytest

from paper_2505_00448_gb300 import dist as D
from paper_2505_00448_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _cohort():
    return synth.small_cohort(77, n_cont=600, n_cat=300, S=300 + 7, miss=0.2, lev_lo=2, lev_hi=5)


def _part_outputs(coh, test, va, vb, world, rank):
    """The oracle on exactly the entries `rank` owns; other entries NaN / -1."""
    from oracle import oracle as O
    na = len(va)
    nb = na if vb is None else len(vb)
    sym = vb is None
    ii, jj = D.owned_pairs(na, nb, world, rank, sym)
    if sym:                                   # compute i <= j once, mirror
        keep = ii <= jj
        ii, jj = ii[keep], jj[keep]
    stat = np.full((na, nb), np.nan)
    p = np.full((na, nb), np.nan)
    n = np.full((na, nb), -1, np.int32)
    pa = np.asarray(va)[ii]
    pb = (np.asarray(va) if sym else np.asarray(vb))[jj]
    s_, p_, n_ = O.run_pairs(test, coh["X"], coh["missing"], coh["vtype"], coh["nlev"], pa, pb)
    for a, b in ((ii, jj), (jj, ii)) if sym else ((ii, jj),):
        stat[a, b], p[a, b], n[a, b] = s_, p_, n_
    return {"stat": stat, "p": p, "n": n}


def _worker(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {"max": D.max_over_ranks(10.0 + 5.0 * rank, dist), "sum": D.sum_over_ranks(rank + 1, dist)}
    coh = _cohort()
    blocks = {}
    for test, va, vb in (("pearson", coh["cont"], None), ("anova", coh["cat"], coh["cont"][:40])):
        blocks[test] = _part_outputs(coh, test, va, vb, world, rank)
    res["gathered"] = D.gather_to_root(blocks, dist)
    res["ctxs"] = D.gather_to_root(D.shard_blocks(256, world, rank, block=1), dist)
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(outdir, f"r{rank}.npy"), np.array([res], dtype=object), allow_pickle=True)


def test_world2_gloo_stitched_oracle_blocks(tmp_path):
    from oracle import oracle as O
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "r0.npy", allow_pickle=True)[0]
    r1 = np.load(tmp_path / "r1.npy", allow_pickle=True)[0]
    assert r0["max"] == r1["max"] == 15.0
    assert r0["sum"] == r1["sum"] == 3.0
    assert r1["gathered"] is None
    g = r0["gathered"]
    coh = _cohort()
    for test, va, vb in (("pearson", coh["cont"], None), ("anova", coh["cat"], coh["cont"][:40])):
        full = O.run(test, coh["X"], coh["missing"], coh["vtype"], coh["nlev"], va, vb)
        na = len(va)
        nb = na if vb is None else len(vb)
        for k, ref in zip(("stat", "p", "n"), full):
            got = D.stitch([g[r][test][k] for r in range(world)], na, nb, vb is None)
            assert np.array_equal(got, ref, equal_nan=True), (test, k)
        # each part wrote only its own entries
        own = D.owner(na, nb, world, vb is None)
        for r in range(world):
            assert (g[r][test]["n"][own != r] == -1).all()
    assert sorted(r0["ctxs"][0] + r0["ctxs"][1]) == list(range(256))


def test_split_rule_covers_once_and_balances():
    for world in (1, 2, 3, 4, 8):
        for n in (1, 255, 256, 600, 4000, 10000):
            own = D.part_of_row(np.arange(n), world)
            assert own.min() >= 0 and own.max() < world
            # every row has exactly one part; blocks of 256 stay whole
            assert all(len(set(own[b:b + 256])) == 1 for b in range(0, n, 256))
            rows = [D.owned_rows(n, world, r) for r in range(world)]
            assert sorted(np.concatenate(rows).tolist()) == list(range(n))
        # upper-triangle work per part within 15% of the mean once every part has
        # two rounds of blocks (4,000 rows: 16 blocks)
        if world <= 8:
            n = 4000
            w = np.array([sum(n - i for i in D.owned_rows(n, world, r)) for r in range(world)], float)
            assert w.max() / w.mean() < 1.15, (world, w)
    o = D.owner(5, 5, 3, True)
    assert (o == o.T).all()
    with pytest.raises(ValueError):
        D.owned_rows(10, 2, 2)


def test_context_shards_and_split_value():
    for world in (1, 2, 3, 4, 8):
        for n, block in ((0, 1), (7, 1), (256, 1), (1000, 8), (37, 5)):
            parts = [D.shard_blocks(n, world, r, block) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert sorted(flat) == list(range(n)) and len(flat) == n
    with pytest.raises(ValueError):
        D.shard_blocks(10, 2, 2)
    # the split's throughput: all units over the slowest rank's time (no replica factor)
    assert D.split_value(100, 2.0) == 50.0
