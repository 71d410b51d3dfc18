"""Multi-GPU bookkeeping for one node: one process per GPU (torchrun), no
collective on the data path. The pairs of an all-pairs test are independent,
so work is split across ranks and only timings (and, when wanted, the output
blocks) are combined: block-cyclic shards of the upper-triangle tile list or of
a batch's sample contexts, the slowest rank's step time, and a host gather.
Works with the NCCL backend (GPU tensors) and with gloo (CPU tensors, tests)."""
from __future__ import annotations

import os


def env_ranks():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 if absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _tensor(x, dist):
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    return torch.tensor([float(x)], dtype=torch.float64, device=dev)


def max_over_ranks(x, dist=None):
    """The largest of every rank's value (every rank gets it)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = _tensor(x, dist)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist=None):
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = _tensor(x, dist)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_blocks(n_items, world, rank, block=1):
    """Indices of rank's share of n_items, dealt out in blocks of `block`
    consecutive items round-robin over the ranks (block-cyclic)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank")
    out = []
    for b0 in range(block * rank, n_items, block * world):
        out.extend(range(b0, min(n_items, b0 + block)))
    return out


def triangle_tiles(n_rows, tile):
    """Tile pairs (I, J), I <= J, of the upper triangle of an n_rows x n_rows output."""
    t = -(-n_rows // tile)
    return [(i, j) for i in range(t) for j in range(i, t)]


def shard_triangle(n_rows, tile, world, rank, block=8):
    """Rank's tiles of the upper triangle, block-cyclic over the row-major tile list
    (neighbouring tiles share operand rows, so blocks keep some reuse per rank)."""
    tiles = triangle_tiles(n_rows, tile)
    return [tiles[k] for k in shard_blocks(len(tiles), world, rank, block)]


def gather_to_root(obj, dist=None, root=0):
    """Every rank's object, in rank order, on the root rank (None elsewhere)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == root else None
    dist.gather_object(obj, out, dst=root)
    return out


def weak_scaling_value(units_per_rank, seconds_slowest, world):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds_slowest
