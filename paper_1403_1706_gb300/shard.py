"""Read sharding across ranks: one process per GPU, each mapping a disjoint slice of the reads.

A read's hits depend only on the read, its budget k and the reference, never on the other reads
of its batch, so the mapping partitions by read with no exchange step: every rank holds its own
resident copy of the packed reference and maps its slice (weak scaling).  The only cross-rank
traffic is host bookkeeping: the maximum of the ranks' step times for throughput, the total of
the reads they mapped, and, when one caller wants a single result set, a gather of the per-rank
results renumbered to global read ids.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n_reads: int, world: int, rank: int) -> tuple[int, int]:
    """The contiguous read range [a, b) of `rank`; sizes differ by at most one read."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} out of range for world size {world}")
    if n_reads < 0:
        raise ValueError("negative read count")
    base, extra = divmod(n_reads, world)
    a = rank * base + min(rank, extra)
    return a, a + base + (1 if rank < extra else 0)


def merge_rank_hits(parts):
    """Concatenate per-rank results into one result set with global read ids.

    `parts` is a sequence of (first_read, read, strand, end, dist) in rank order, each rank's
    arrays sorted by (read, strand, end) with read ids local to its shard.  Shards are contiguous
    and ascending, so offsetting the ids and concatenating keeps the global order.
    """
    reads, strands, ends, dists = [], [], [], []
    last = -1
    for first, r, s, e, d in parts:
        r = np.asarray(r, dtype=np.uint64) + np.uint64(first)
        if r.size:
            if int(r[0]) <= last:
                raise ValueError("rank parts are not in ascending read order")
            last = int(r[-1])
        reads.append(r.astype(np.uint32))
        strands.append(np.asarray(s, dtype=np.uint8))
        ends.append(np.asarray(e, dtype=np.int64))
        dists.append(np.asarray(d, dtype=np.int32))
    cat = (lambda xs, dt: np.concatenate(xs) if xs else np.zeros(0, dt))
    return (cat(reads, np.uint32), cat(strands, np.uint8), cat(ends, np.int64), cat(dists, np.int32))


def _reduce(x: float, op, device):
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    """The largest of the ranks' values (a step time); the value itself without a process group."""
    import torch.distributed as dist
    return _reduce(float(x), dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device=None) -> float:
    """The total of the ranks' values (reads mapped); the value itself without a process group."""
    import torch.distributed as dist
    return _reduce(float(x), dist.ReduceOp.SUM, device)
