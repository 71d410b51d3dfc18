"""Multi-GPU bookkeeping for one node: one process per GPU (torchrun), no
collective on the data path. The pairs of an all-pairs test are independent
(Sec. 3.5.1), so a call is split over the ranks by napg_run_part: output rows
in blocks of PART_ROWS, dealt to the parts back and forth so that a triangle's
long and short rows pair up; each rank computes the pairs of its rows and the
output blocks are gathered afterwards. This module holds the same ownership
rule as the library (for stitching and for tests), the slowest rank's time,
the split throughput, and a host gather. Works with the NCCL backend (GPU
tensors) and with gloo (CPU tensors, tests)."""
from __future__ import annotations

import os

import numpy as np

PART_ROWS = 256     # NAPG_PART_ROWS


def env_ranks():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 if absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def part_of_row(row, nparts):
    """The part that owns output row `row`: block b = row // PART_ROWS goes to
    b mod nparts in even rounds b // nparts and to nparts - 1 - (b mod nparts)
    in odd ones."""
    b = np.asarray(row) // PART_ROWS
    r, k = b // nparts, b % nparts
    return np.where(r % 2 == 1, nparts - 1 - k, k)


def owned_rows(n_rows, nparts, part):
    """The output rows of `part`."""
    if nparts < 1 or not 0 <= part < nparts:
        raise ValueError("bad part")
    rows = np.arange(n_rows)
    return rows[part_of_row(rows, nparts) == part]


def owner(n_a, n_b, nparts, symmetric):
    """Owner of every output entry: the owner of row min(i, j) for a symmetric
    call (pairs i <= j are computed for owned rows i and mirrored), of row i for
    an A x B call."""
    i = np.arange(n_a)[:, None]
    j = np.arange(n_b)[None, :]
    return part_of_row(np.minimum(i, j) if symmetric else np.broadcast_to(i, (n_a, n_b)), nparts)


def owned_pairs(n_a, n_b, nparts, part, symmetric):
    """(rows, cols) of the entries `part` writes."""
    return np.nonzero(owner(n_a, n_b, nparts, symmetric) == part)


def stitch(parts, n_a, n_b, symmetric):
    """One output from every part's output (parts[k] written by part k): each
    entry taken from its owner."""
    own = owner(n_a, n_b, len(parts), symmetric)
    out = np.array(parts[0], copy=True)
    for k in range(1, len(parts)):
        sel = own == k
        out[sel] = np.asarray(parts[k])[sel]
    return out


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
    consecutive items round-robin over the ranks (block-cyclic): the sample
    contexts of a batch."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank")
    out = []
    for b0 in range(block * rank, n_items, block * world):
        out.extend(range(b0, min(n_items, b0 + block)))
    return out


def gather_to_root(obj, dist=None, root=0):
    """Every rank's object, in rank order, on the root rank (None elsewhere)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size() if dist.get_rank() == root else None
    dist.gather_object(obj, out, dst=root)
    return out


def split_value(total_units, seconds_slowest):
    """Whole-job throughput of a split call: all units (every rank's share) over
    the slowest rank's time."""
    return total_units / seconds_slowest
