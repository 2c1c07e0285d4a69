"""Parity at the workloads' full sizes, in the launch configuration the bench times.

The GPU maps whole batches; the oracle checks a sample of reads one by one against the whole
reference (exact hit sets; a read's hits do not depend on the other reads of its batch).  On the
3.1 Gbp workload a property that holds at any size is checked as well: every planted read's true
end lies in a run of ends within k edits whose canonical tuple (found here by a local DP window
of the oracle) must be in the GPU output.  The postprocessing of that batch (starts, ranks,
qualities, extended CIGARs) is checked hit by hit for a sample of reads, the oracle annotating and
aligning the GPU's own hit lists of those reads.
"""
from concurrent.futures import ThreadPoolExecutor

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


def has_short_period_stretch(read: np.ndarray, length: int = 16, pmax: int = 3) -> bool:
    """True if some `length`-base stretch of the read repeats with a period of at most `pmax`
    bases (a poly-A, dinucleotide or trinucleotide run)."""
    r = np.asarray(read, dtype=np.uint8)
    for P in range(1, pmax + 1):
        w = length - P
        if r.size < length:
            break
        bad = np.concatenate([[0], np.cumsum(r[P:] != r[:-P])])
        if np.any(bad[w:] - bad[:-w] == 0):
            return True
    return False


def oracle_jobs(ref, jobs, parts, workers=14):
    """oracle.map_filter for every job (reads, k, q, mode), each split into `parts` slices of its
    reads, all side by side in threads (ctypes releases the GIL; a read's hits do not depend on the
    other reads); returns each job's hit set in read order."""
    tasks = []
    for j, (sub, k, q, mode) in enumerate(jobs):
        bounds = np.linspace(0, sub.n, parts + 1).astype(int)
        for a, b in zip(bounds[:-1], bounds[1:]):
            if b > a:
                tasks.append((j, a, b))

    def run(t):
        j, a, b = t
        sub, k, q, mode = jobs[j]
        kk = np.ascontiguousarray(np.asarray(k)[a:b]) if np.ndim(k) else k
        sl = sub.slice(a, b)
        h = oracle.map_filter(ref, sl.seq, sl.offsets, kk, q, mode)
        h["read"] += np.uint32(a)
        return j, h
    with ThreadPoolExecutor(min(workers, len(tasks))) as ex:
        res = list(ex.map(run, tasks))
    return [oracle.sort_hits(np.concatenate([h for jj, h in res if jj == j])) for j in range(len(jobs))]


@pytest.fixture(scope="module")
def human_ref(gpu):
    w = synth.WORKLOADS["human_3g1_10m"]
    ref = synth.make_reference(w["ref_len"], 1403, w["repeat_frac"], w["tandem_frac"])
    return ref, gpu.pack_reference(ref)


@pytest.fixture(scope="module")
def human_batch(gpu, human_ref):
    """The first 2^20-read batch of the 3.1 Gbp workload (bench seed), mapped on the GPU in both
    modes with the bench's q = 16, k = 5."""
    ref, R = human_ref
    w = synth.WORKLOADS["human_3g1_10m"]
    seed = 1706 + list(synth.WORKLOADS).index("human_3g1_10m")
    reads = synth.make_reads(ref, 1 << 20, seed, lengths=w["lengths"], rate_range=w["rate_range"],
                             random_frac=w["random_frac"])
    B = gpu.index_reads(R, reads.seq, reads.offsets, 16, k=5)
    h = gpu.map(R, B, "all")
    st = gpu.get_map_stats(B)
    hb = gpu.map(R, B, "best")
    thr, lowcx = gpu.export_read_params(B)
    B.free()
    return ref, reads, h, hb, lowcx, st


def test_human_scale_batch_sampled_exact(human_batch):
    """2,000 evenly spaced reads of the batch plus 150 of the reads the GPU verified around
    frequent-q-gram clusters, exact against the oracle in both modes.  The low-complexity sample
    leaves out reads holding a 16-base stretch of period 1-3: against 3.1 Gbp a poly-A read has
    ~2e8 q-gram hits per strand, more than the oracle's per-diagonal lists hold; those reads are
    checked exactly at 7 Mbp (test_gpu_lowcx_paths) and 2 Mbp (test_repeat_rich_scaled)."""
    ref, reads, h, hb, lowcx, st = human_batch
    assert st["lowcx_rest_segments"] > 0 and st["lowcx_reads"] > 5000
    even = np.unique(np.linspace(0, reads.n - 1, 2000).astype(np.int64))
    rng = np.random.default_rng(11)
    lc = [int(r) for r in rng.permutation(np.flatnonzero(lowcx)) if not has_short_period_stretch(
        np.frombuffer(reads.read(int(r)), np.uint8))][:150]
    assert len(lc) == 150
    idx = np.unique(np.concatenate([even, np.asarray(lc, np.int64)]))
    sub = reads.subset(idx)
    wants = oracle_jobs(ref, [(sub, 5, 16, "all"), (sub, 5, 16, "best")], 7)
    for mode, got, want in (("all", h, wants[0]), ("best", hb, wants[1])):
        assert np.array_equal(_hits_of(got, idx), want), mode


def test_uneven_human_scale_engine_sampled_exact(gpu, human_ref):
    """The uneven configuration on the 3.1 Gbp reference: 2^17 reads of 50, 75, 100, 150 and
    250 bp (2 % errors, k = ceil(0.05 L)) in one engine submission, autotuned as in the bench;
    2,000 evenly spaced reads (without 16-base stretches of period 1-3, as above) exact against
    the oracle, each length class at the largest q its reads admit."""
    ref, R = human_ref
    w = synth.WORKLOADS["uneven_3g1_10m"]
    reads = synth.make_reads(ref, 1 << 17, 4242, lengths=w["lengths"], rate_range=w["rate_range"],
                             random_frac=0.0)
    E = gpu.Engine(R, k_permille=50, executors=2, autotune=True)
    try:
        got = {m: E.wait(E.submit(reads.seq, reads.offsets, m)) for m in ("all", "best")}
    finally:
        E.free()
    even = np.unique(np.linspace(0, reads.n - 1, 2000).astype(np.int64))
    idx = np.asarray([int(r) for r in even if not has_short_period_stretch(
        np.frombuffer(reads.read(int(r)), np.uint8))], np.int64)
    assert idx.size > 1900
    lens = reads.lengths[idx]
    jobs, sels = [], []
    for mode in ("all", "best"):
        for q, sel in ((12, lens == 50), (15, lens == 75), (16, lens >= 100)):
            sub = reads.subset(idx[sel])
            jobs.append((sub, synth.k_of_length(sub.lengths, "5pct"), q, mode))
            sels.append(idx[sel])
    res = oracle_jobs(ref, jobs, 2)
    for x, mode in enumerate(("all", "best")):
        parts = []
        for y in range(3):
            want = res[3 * x + y]
            want["read"] = sels[3 * x + y][want["read"]]
            parts.append(want)
        want = oracle.sort_hits(np.concatenate(parts))
        g = got[mode]
        keep = np.isin(g["read"], idx.astype(np.uint32))
        gg = oracle.sort_hits(g[keep].astype(oracle.HIT_DTYPE))
        assert np.array_equal(gg, want), mode


def test_human_scale_batch_properties(human_batch):
    ref, reads, h, hb, lowcx, st = human_batch
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


def _postprocessing_sample(gpu, ref, R, reads, n_sample=2000, max_hits=4000):
    """Maps one batch (q = 16, stride 16, k = 5, all hits), runs the whole postprocessing on the GPU (starts,
    ranks, qualities, extended CIGARs of every hit), and checks it against the oracle for
    n_sample evenly spaced reads with at most max_hits hits each (the oracle's rank is quadratic
    in a read's hits): the oracle annotates and aligns the GPU's own hit lists of those reads.
    Returns the number of hits checked."""
    import torch
    B = gpu.index_reads(R, reads.seq, reads.offsets, 16, k=5, stride=16)
    try:
        dh = gpu.map_device(R, B, "all")
        h = dh.to_numpy()
        start, rank, mapq = gpu.annotate_hits(R, B, dh)
        ops, nops = gpu.hit_alignments(R, B, dh, start)
        per_read = np.bincount(h["read"].astype(np.int64), minlength=reads.n)
        cand = np.flatnonzero((per_read > 0) & (per_read <= max_hits))
        idx = cand[np.unique(np.linspace(0, cand.size - 1, n_sample).astype(np.int64))]
        sel = np.flatnonzero(np.isin(h["read"], idx.astype(np.uint32)))
        sub = reads.subset(idx)
        pos = np.full(reads.n, -1, np.int64)
        pos[idx] = np.arange(idx.size)
        hs = h[sel].copy()
        hs["read"] = pos[hs["read"].astype(np.int64)].astype(np.uint32)
        ws, wr, wq = oracle.annotate(ref, sub.seq, sub.offsets, hs)
        assert np.array_equal(start.cpu().numpy()[sel], ws)
        assert np.array_equal(rank.cpu().numpy()[sel].astype(np.uint32), wr)
        assert np.array_equal(mapq.cpu().numpy()[sel].astype(np.int32), wq)
        t = torch.as_tensor(sel, dtype=torch.int64, device=ops.device)
        got = gpu.cigars(ops[t], nops[t])
        exp = oracle.alignments(ref, sub.seq, sub.offsets, hs, ws)
        bad = [(int(sel[x]), g, e) for x, (g, e) in enumerate(zip(got, exp)) if g != e]
        assert not bad, bad[:5]
        return int(sel.size)
    finally:
        B.free()


def test_human_scale_postprocessing_sampled_exact(gpu, human_ref):
    """The postprocessing of the bench's first 2^20-read batch of the 3.1 Gbp workload, as
    `bench.py --mode post` runs it: every hit of 2,000 evenly spaced reads among those with at
    most 4,000 hits (starts, ranks, qualities, alignments) exact against the oracle."""
    ref, R = human_ref
    w = synth.WORKLOADS["human_3g1_10m"]
    seed = 1706 + list(synth.WORKLOADS).index("human_3g1_10m")
    reads = synth.make_reads(ref, 1 << 20, seed, lengths=w["lengths"], rate_range=w["rate_range"],
                             random_frac=w["random_frac"])
    assert _postprocessing_sample(gpu, ref, R, reads) > 4_000
