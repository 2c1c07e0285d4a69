"""The N > 1 path on CPU: two gloo ranks shard a read set, map their slices, and the merged
result equals mapping the whole set in one process; the timing reductions are max / sum over
ranks.  The oracle stands in for the GPU mapping (a read's hits do not depend on its batch)."""
import os
import socket
import tempfile

import numpy as np
import pytest

import oracle
import synth
from paper_1403_1706_gb300 import shard


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    ref = synth.make_reference(120_000, 41, 0.05, 0.01)
    reads = synth.make_reads(ref, 301, 43, lengths=(100,), rate_range=(0.01, 0.04), random_frac=0.05)
    return ref, reads


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ref, reads = _workload()
        a, b = shard.shard_bounds(reads.n, world, rank)
        sub = reads.slice(a, b)
        h = oracle.map_filter(ref, sub.seq, sub.offsets, 5, 11, "all")
        parts = [None] * world
        dist.all_gather_object(parts, (a, h["read"], h["strand"], h["end"], h["dist"]))
        t_max = shard.max_over_ranks(10.0 + rank)
        n_tot = shard.sum_over_ranks(b - a)
        if rank == 0:
            r, s, e, d = shard.merge_rank_hits(parts)
            np.savez(os.path.join(outdir, "merged.npz"), read=r, strand=s, end=e, dist=d,
                     t_max=t_max, n_tot=n_tot)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_shard_bounds_partition():
    for n in (0, 1, 7, 1000, 10_000_001):
        for world in (1, 2, 3, 8):
            rs = [shard.shard_bounds(n, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(10, 2, 2)


def test_merge_rejects_out_of_order():
    with pytest.raises(ValueError):
        shard.merge_rank_hits([(5, [0], [0], [1], [0]), (0, [0], [0], [1], [0])])


def test_two_gloo_ranks_match_single_process():
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        z = np.load(os.path.join(d, "merged.npz"))
        ref, reads = _workload()
        want = oracle.map_filter(ref, reads.seq, reads.offsets, 5, 11, "all")
        got = np.zeros(z["read"].size, dtype=oracle.HIT_DTYPE)
        for f in ("read", "strand", "end", "dist"):
            got[f] = z[f]
        assert want.size > reads.n // 2
        assert np.array_equal(got, want)
        assert float(z["t_max"]) == 11.0 and int(z["n_tot"]) == reads.n
