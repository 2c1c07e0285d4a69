"""GPU parity of the alignment of every hit (Section "Postprocessing": the actual alignment of each
hit) against the oracle (oracle_cigar: the pattern against its reference bases, both ends fixed,
traced back preferring the diagonal, then reference-only, then read-only steps).  The oracle
aligns its own hit list with its own starts, which the GPU's must equal first; the extended
CIGAR strings are then compared hit by hit: the hand example, repeat-rich reads with many hits
on both strands, reads of 50-250 bp with per-read budgets (up to 13 edits), and a reference of
several contigs with gaps of N and reads holding N.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _check(gpu, R, ref, seq, offs, q, mode, k=None, k_permille=None, segments=None, prepared=None):
    B = gpu.index_reads(R, seq, offs, q, k=k, k_permille=k_permille)
    dh = gpu.map_device(R, B, mode)
    lens = np.diff(np.asarray(offs, np.int64))
    kv = np.full(lens.size, k) if k is not None else (lens * k_permille + 999) // 1000
    rseq = seq if prepared is None else prepared
    want = oracle.map_filter(ref, rseq, offs, kv, q, mode, segments=segments)
    assert np.array_equal(dh.to_numpy(), want)
    start, _, _ = gpu.annotate_hits(R, B, dh)
    ws, _, _ = oracle.annotate(ref, rseq, offs, want, segments=segments)
    assert np.array_equal(start.cpu().numpy(), ws)
    ops, nops = gpu.hit_alignments(R, B, dh, start)
    got = gpu.cigars(ops, nops)
    exp = oracle.alignments(ref, rseq, offs, want, ws)
    bad = [(i, g, e) for i, (g, e) in enumerate(zip(got, exp)) if g != e]
    assert not bad, bad[:5]
    B.free()
    return got


def test_hand_example(gpu):
    R = gpu.pack_reference(b"TTACGTTACGATT")
    got = _check(gpu, R, b"TTACGTTACGATT", b"ACGTA", [0, 5], 2, "all", k=1)
    assert got == ["4=1I", "3=1I1=", "5=", "4=1I"]


@pytest.mark.parametrize("mode", ["all", "best"])
def test_repeat_rich_reads(gpu, mode):
    ref, reads, w = synth.make_workload("repeat_100mbp_1m", ref_len=1_000_000, n_reads=2000)
    R = gpu.pack_reference(ref)
    got = _check(gpu, R, ref, reads.seq, reads.offsets, 16, mode, k=5)
    assert len(got) > 1500 and any("I" in c or "D" in c for c in got) and any("X" in c for c in got)


def test_uneven_lengths_and_budgets(gpu):
    ref, reads, w = synth.make_workload("uneven_3g1_10m", ref_len=500_000, n_reads=1500)
    R = gpu.pack_reference(ref)
    got = _check(gpu, R, ref, reads.seq, reads.offsets, 12, "all", k_permille=50)
    assert max(len(c) for c in got) > 10


def test_contigs_and_unknown_bases(gpu):
    raw = synth.make_reference(300_000, 21, repeat_frac=0.1).copy()
    raw[100_000:100_050] = ord("N")
    raw[180_000:180_005] = ord("N")
    contigs = [0, 150_000]
    text, seg = oracle.prepare_reference(raw, contigs, gap_min=16, seed=4)
    reads = synth.make_reads(text, 1000, 22, lengths=(100, 150), rate_range=(0.0, 0.04))
    seq = reads.seq.copy()
    seq[reads.offsets[1:-1:7].astype(np.int64)] = ord("N")
    prepared = oracle.prepare_reads(seq, reads.offsets, seed=4)
    R = gpu.pack_reference(raw, contigs=contigs, seed=4)
    _check(gpu, R, text, seq, reads.offsets, 16, "all", k=5, segments=seg, prepared=prepared)


def test_too_few_ops_per_hit_is_refused(gpu):
    ref = synth.make_reference(50_000, 5)
    reads = synth.make_reads(ref, 200, 6, lengths=(100,), rate_range=(0.03, 0.05))
    R = gpu.pack_reference(ref)
    B = gpu.index_reads(R, reads.seq, reads.offsets, 16, k=5)
    dh = gpu.map_device(R, B, "all")
    start, _, _ = gpu.annotate_hits(R, B, dh)
    assert dh.n > 100
    with pytest.raises(gpu.PeanutError):
        gpu.hit_alignments(R, B, dh, start, ops_per_hit=1)  # a hit with an edit has 2 or more runs
    ops, nops = gpu.hit_alignments(R, B, dh, start)
    assert int(nops.max()) <= 11
    ops2, nops2 = gpu.hit_alignments(R, B, dh, start)  # the same again: the scratch is fresh each call
    assert np.array_equal(nops.cpu().numpy(), nops2.cpu().numpy())
    n = nops.cpu().numpy()
    o1, o2 = ops.cpu().numpy(), ops2.cpu().numpy()
    assert all(np.array_equal(o1[x, :n[x]], o2[x, :n[x]]) for x in range(n.size))
    B.free()


def test_every_distance_class_and_the_reference_ends(gpu):
    """Reads of 200 bases with 0 to 10 edits (k = 10), placed at the very start and end of the
    reference as well as inside it, so that distances 0-3, 4-7 and 8-10 (the three band widths of
    the kernels) all occur, and bands that begin before position 0 or end at the last base."""
    rng = np.random.default_rng(31)
    ref = synth.make_reference(20_000, 32)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    reads = []
    for x in range(300):
        p = 0 if x % 5 == 0 else (ref.size - 200 if x % 5 == 1 else int(rng.integers(0, ref.size - 200)))
        r = list(ref[p:p + 200])
        for _ in range(x % 11):
            y = int(rng.integers(0, len(r)))
            op = rng.random()
            if op < 0.5:
                r[y] = acgt[(list(acgt).index(r[y]) + 1) % 4]
            elif op < 0.75:
                r.insert(y, acgt[int(rng.integers(0, 4))])
            else:
                del r[y]
        reads.append(np.array(r[:200], np.uint8))
    offs = np.concatenate([[0], np.cumsum([r.size for r in reads])]).astype(np.int64)
    seq = np.concatenate(reads)
    R = gpu.pack_reference(ref)
    got = _check(gpu, R, ref, seq, offs, 16, "all", k=10)
    h = oracle.map_filter(ref, seq, offs, 10, 16, "all")
    d = h["dist"]
    assert (d <= 3).any() and ((d >= 4) & (d <= 7)).any() and (d >= 8).any(), np.bincount(d)
    st, _, _ = oracle.annotate(ref, seq, offs, h)
    assert (st == 0).any() and (h["end"] == ref.size - 1).any()
    assert len(got) == len(h)
