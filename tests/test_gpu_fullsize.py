"""Parity at the workloads' full sizes, in the launch configuration the bench times.

The GPU maps whole batches; the oracle checks a sample of reads one by one against the whole
reference (exact hit sets; a read's hits do not depend on the other reads of its batch).  On the
3.1 Gbp workload a property that holds at any size is checked as well: every planted read's true
end lies in a run of ends within k edits whose canonical tuple (found here by a local DP window
of the oracle) must be in the GPU output.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _hits_of(h, idx):
    """GPU hits of the reads idx (sorted), renumbered 0..len(idx)-1."""
    pos = {int(r): i for i, r in enumerate(idx)}
    keep = np.isin(h["read"], np.asarray(idx, dtype=np.uint32))
    out = h[keep].copy()
    out["read"] = [pos[int(r)] for r in out["read"]]
    return oracle.sort_hits(out)


def test_repeat_rich_full_size_sampled(gpu):
    ref, reads, w = synth.make_workload("repeat_100mbp_1m")
    R = gpu.pack_reference(ref)
    B = gpu.index_reads(R, reads.seq, reads.offsets, 16, k=5)
    idx = np.arange(0, reads.n, reads.n // 200)[:200]
    sub = reads.subset(idx)
    for mode in ("all", "best"):
        got = _hits_of(gpu.map(R, B, mode), idx)
        want = oracle.map_filter(ref, sub.seq, sub.offsets, 5, 16, mode)
        assert np.array_equal(got, want), mode


@pytest.fixture(scope="module")
def human_batch(gpu):
    """The first 2^20-read batch of the 3.1 Gbp workload (bench seed), mapped on the GPU."""
    w = synth.WORKLOADS["human_3g1_10m"]
    ref = synth.make_reference(w["ref_len"], 1403, w["repeat_frac"], w["tandem_frac"])
    seed = 1706 + list(synth.WORKLOADS).index("human_3g1_10m")
    reads = synth.make_reads(ref, 1 << 20, seed, lengths=w["lengths"], rate_range=w["rate_range"],
                             random_frac=w["random_frac"])
    R = gpu.pack_reference(ref)
    B = gpu.index_reads(R, reads.seq, reads.offsets, 16, k=5)
    h = gpu.map(R, B, "all")
    return ref, reads, h


def test_human_scale_batch_sampled_exact(human_batch):
    ref, reads, h = human_batch
    idx = np.arange(0, reads.n, reads.n // 8)[:8]
    sub = reads.subset(idx)
    want = oracle.map_filter(ref, sub.seq, sub.offsets, 5, 16, "all")
    assert np.array_equal(_hits_of(h, idx), want)


def test_human_scale_batch_properties(human_batch):
    ref, reads, h = human_batch
    k = 5
    # sorted by (read, strand, end), unique, within budget
    key = h["read"].astype(np.int64) * 2 + h["strand"]
    assert np.all((np.diff(key) > 0) | ((np.diff(key) == 0) & (np.diff(h["end"]) > 0)))
    assert h["dist"].max() <= k and h["read"].max() < reads.n
    got = set(zip(h["read"].tolist(), h["strand"].tolist(), h["end"].tolist(), h["dist"].tolist()))
    # planted reads: the canonical tuple of the run holding the true end (local DP window)
    rng = np.random.default_rng(7)
    planted = np.flatnonzero((reads.truth_edits >= 0) & (reads.truth_edits <= k))
    checked = 0
    for r in rng.choice(planted, 500, replace=False):
        s = int(reads.truth_strand[r])
        read = reads.read(int(r))
        pat = read if s == 0 else synth.revcomp_ascii(read).tobytes()
        m = len(pat)
        e = int(reads.truth_end[r])
        lo, hi = max(0, e - 600), min(ref.size, e + 600)
        D = oracle.semiglobal_column(pat, ref[lo:hi])
        exact_from = (0 if lo == 0 else m + k - 1)  # window values <= k are exact from here on
        j = e - lo
        assert D[j] <= k, (r, D[j])
        a = j
        while a - 1 >= 0 and D[a - 1] <= k:
            a -= 1
        b = j
        while b + 1 < D.size and D[b + 1] <= k:
            b += 1
        if a - 1 < exact_from or b + 1 >= D.size:
            continue  # the run is not fully inside the window
        run = D[a:b + 1]
        jstar = a + int(np.argmin(run))
        assert (int(r), s, lo + jstar, int(run.min())) in got, int(r)
        checked += 1
    assert checked > 450


def test_reference_beyond_2_32_bases(gpu):
    """A 4.4 Gbp reference (positions past 2^32: the block paths sort 41-bit keys).  The same reads
    mapped at q = 14 (~3,000 hits per read: block window path) and at q = 16 (warp path), with
    the default and a small frequency cap, must give one hit set; planted reads keep the
    canonical tuple of the run holding their true end (local DP window of the oracle)."""
    n = 4_400_000_000
    ref = synth.make_reference(n, 2718, 0.45, 0.01)
    reads = synth.make_reads(ref, 20000, 2719, lengths=(100,), rate_range=(0.01, 0.04), random_frac=0.05)
    R = gpu.pack_reference(ref)
    sets = []
    for q, cap in ((16, 0), (14, 0), (14, 128)):  # a 14-gram occurs ~33 times by chance here
        B = gpu.index_reads(R, reads.seq, reads.offsets, q, k=5, freq_cap=cap)
        sets.append(gpu.map(R, B, "all"))
        st = gpu.get_map_stats(B)
        if q == 14:
            assert st["med_reads"] > reads.n // 2
        B.free()
    assert np.array_equal(sets[0], sets[1]) and np.array_equal(sets[0], sets[2])
    h = sets[0]
    assert h["end"].max() >= 1 << 32 or (reads.truth_end >= 1 << 32).sum() == 0
    got = set(zip(h["read"].tolist(), h["strand"].tolist(), h["end"].tolist(), h["dist"].tolist()))
    k = 5
    rng = np.random.default_rng(3)
    planted = np.flatnonzero((reads.truth_edits >= 0) & (reads.truth_edits <= k) & (reads.truth_end >= 1 << 32))
    checked = 0
    for r in rng.choice(planted, min(100, planted.size), replace=False):
        s = int(reads.truth_strand[r])
        read = reads.read(int(r))
        pat = read if s == 0 else synth.revcomp_ascii(read).tobytes()
        m = len(pat)
        e = int(reads.truth_end[r])
        lo, hi = max(0, e - 600), min(ref.size, e + 600)
        D = oracle.semiglobal_column(pat, ref[lo:hi])
        j = e - lo
        assert D[j] <= k
        a = j
        while a - 1 >= 0 and D[a - 1] <= k:
            a -= 1
        b = j
        while b + 1 < D.size and D[b + 1] <= k:
            b += 1
        if a - 1 < m + k - 1 or b + 1 >= D.size:
            continue
        run = D[a:b + 1]
        assert (int(r), s, lo + a + int(np.argmin(run)), int(run.min())) in got, int(r)
        checked += 1
    assert checked > 80
