"""GPU parity on references of several contigs with unknown bases, and on reads with N.

Section "Overview": every step runs per chromosome, so no hit spans two contigs; Section "The
q-group index" (encoding paragraph): N becomes a random base and long runs of N stay out of the
index.  The library's reading (seeded replacement, runs of >= gap_min Ns as gaps, segments no
alignment leaves) is compared element by element with the oracle's (pinned in
test_oracle_contigs.py): the segment list, the hit sets in both modes (scan, sampled scan,
reference-side index, engine), and the postprocessing.  The reference mixes contigs of unequal
length, gaps inside contigs and at their ends, short N runs that stay in the index, soft-masked
(lower-case) stretches and a repeat family copied across contigs; reads straddle every boundary
and some carry Ns or are lower-case.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

K, Q, SEED, GAP_MIN = 5, 16, 20140305, 16


def _lower(a):
    return np.where((a >= 65) & (a <= 90), a + 32, a).astype(np.uint8)


def _genome(seed=3):
    rng = np.random.default_rng(seed)
    lens = [400_000, 120_000, 900_000, 250_000, 30_000]
    parts, starts, pos = [], [], 0
    family = synth.make_reference(600, seed + 100)
    for c, L in enumerate(lens):
        a = synth.make_reference(L, seed * 10 + c, repeat_frac=0.05, tandem_frac=0.01).copy()
        a[L // 3:L // 3 + 600] = family  # a repeat that straddles nothing but occurs in every contig
        for _ in range(4):  # gaps (>= gap_min) and short runs (< gap_min) inside the contig
            x = int(rng.integers(0, L - 3000))
            a[x:x + int(rng.integers(GAP_MIN, 2000))] = ord("N")
            y = int(rng.integers(0, L - 20))
            a[y:y + int(rng.integers(1, GAP_MIN))] = ord("N")
        if c == 1:
            a[:500] = ord("N")      # a gap at a contig start
        if c == 3:
            a[-700:] = ord("N")     # a gap at a contig end
        z = int(rng.integers(0, L - 5000))
        a[z:z + 5000] = _lower(a[z:z + 5000])  # soft-masked
        parts.append(a)
        starts.append(pos)
        pos += L
    return np.concatenate(parts), starts


def _reads(text, starts, seg, n, seed):
    """Reads from the prepared text: a third straddle a contig or gap edge, a fifth carry 1-3 Ns,
    a tenth are lower-case."""
    rng = np.random.default_rng(seed)
    edges = sorted(set(starts[1:]) | set(seg[:, 0].tolist()) | set(seg[:, 1].tolist()))
    edges = [e for e in edges if 120 < e < len(text) - 120]
    src = synth.make_reads(text, n, seed, lengths=(100,), rate_range=(0.0, 0.03))
    reads = []
    for i in range(n):
        if i % 3 == 0:
            e = edges[int(rng.integers(0, len(edges)))]
            p = e - int(rng.integers(5, 95))
            r = text[p:p + 100].copy()
            for _ in range(int(rng.integers(0, 3))):
                r[int(rng.integers(0, 100))] = np.frombuffer(b"ACGT", np.uint8)[int(rng.integers(0, 4))]
        else:
            r = np.frombuffer(src.read(i), np.uint8).copy()
        if i % 5 == 1:
            r[rng.integers(0, r.size, int(rng.integers(1, 4)))] = ord("N")
        if i % 10 == 7:
            r = _lower(r)
        reads.append(r)
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum([r.size for r in reads])
    return np.concatenate(reads), offs


@pytest.fixture(scope="module")
def world(gpu):
    raw, starts = _genome()
    text, seg = oracle.prepare_reference(raw, starts, gap_min=GAP_MIN, seed=SEED)
    seq, offs = _reads(text, starts, seg, 3000, 11)
    prepared = oracle.prepare_reads(seq, offs, seed=SEED)
    R = gpu.pack_reference(raw, contigs=starts, gap_min=GAP_MIN, seed=SEED)
    want = {m: oracle.map_filter(text, prepared, offs, K, Q, m, segments=seg) for m in ("all", "best")}
    return raw, starts, text, seg, seq, offs, prepared, R, want


def _same(got, want):
    if not np.array_equal(got, want):
        g, w = set(map(tuple, got.tolist())), set(map(tuple, want.tolist()))
        raise AssertionError(f"{len(got)} vs {len(want)}: missing {sorted(w - g)[:6]}, extra {sorted(g - w)[:6]}")


def test_segments_equal_oracle(gpu, world):
    raw, starts, text, seg, *_ , R, want = world
    got = gpu.ref_segments(R)
    assert np.array_equal(got.astype(np.int64), seg)
    assert len(seg) > len(starts) + 10  # the gaps cut the contigs


@pytest.mark.parametrize("mode", ["all", "best"])
@pytest.mark.parametrize("stride", [1, 4])
def test_map_equals_oracle(gpu, world, mode, stride):
    raw, starts, text, seg, seq, offs, prepared, R, want = world
    B = gpu.index_reads(R, seq, offs, Q, k=K, stride=stride)
    got = gpu.map(R, B, mode)
    B.free()
    _same(got, want[mode])
    assert len(want[mode]) > 1500
    # no hit ends in a gap, and the straddling reads still find their in-segment alignments
    ends = want[mode]["end"]
    x = np.searchsorted(seg[:, 1], ends, side="right")
    assert np.all(seg[x, 0] <= ends)


def test_reference_index_and_engine_equal_oracle(gpu, world):
    raw, starts, text, seg, seq, offs, prepared, R, want = world
    gpu.index_reference(R, Q)
    B = gpu.index_reads(R, seq, offs, Q, k=K, stride=4, ref_index=True)
    _same(gpu.map(R, B, "all"), want["all"])
    B.free()
    E = gpu.Engine(R, k=K, executors=2)
    try:
        t = [E.submit(seq, offs, m) for m in ("all", "best")]
        _same(E.wait(t[0]), want["all"])
        _same(E.wait(t[1]), want["best"])
    finally:
        E.free()


def test_annotation_equals_oracle(gpu, world):
    raw, starts, text, seg, seq, offs, prepared, R, want = world
    B = gpu.index_reads(R, seq, offs, Q, k=K)
    dh = gpu.map_device(R, B, "all")
    h = dh.to_numpy()
    _same(h, want["all"])  # the oracle annotates its own hit list
    start, rank, mapq = gpu.annotate_hits(R, B, dh)
    ws, wr, wq = oracle.annotate(text, prepared, offs, want["all"], segments=seg)
    assert np.array_equal(start.cpu().numpy(), ws)
    assert np.array_equal(rank.cpu().numpy().astype(np.uint32), wr)
    assert np.array_equal(mapq.cpu().numpy().astype(np.int32), wq)
    x = np.searchsorted(seg[:, 1], h["end"], side="right")
    assert np.all(ws >= seg[x, 0])
    B.free()


def test_small_case_equals_bruteforce(gpu):
    """The definition itself (full DP per segment) on a small reference, both modes."""
    raw = synth.make_reference(24_000, 8).copy()
    raw[3000:3040] = ord("N")
    raw[9000:9005] = ord("N")
    raw[:20] = ord("N")
    raw[-30:] = ord("N")
    starts = [0, 6000, 15000, 15100]
    text, seg = oracle.prepare_reference(raw, starts, gap_min=GAP_MIN, seed=5)
    seq, offs = _reads(text, starts, seg, 120, 2)
    prepared = oracle.prepare_reads(seq, offs, seed=5)
    R = gpu.pack_reference(raw, contigs=starts, gap_min=GAP_MIN, seed=5)
    for mode in ("all", "best"):
        want = oracle.map_bruteforce(text, prepared, offs, K, mode, segments=seg)
        B = gpu.index_reads(R, seq, offs, 12, k=K)
        _same(gpu.map(R, B, mode), want)
        B.free()


def test_degenerate_references(gpu):
    """All N (no segment), every N a gap (gap_min 1), a read of Ns only."""
    R = gpu.pack_reference(b"N" * 5000, gap_min=GAP_MIN, seed=1)
    assert gpu.ref_segments(R).shape == (0, 2)
    B = gpu.index_reads(R, b"ACGT" * 25 + b"N" * 100, [0, 100, 200], 12, k=5)
    assert gpu.map(R, B, "all").size == 0
    raw = synth.make_reference(8000, 4).copy()
    raw[100::500] = ord("n")
    text, seg = oracle.prepare_reference(raw, [0, 4000], gap_min=1, seed=9)
    R = gpu.pack_reference(raw, contigs=[0, 4000], gap_min=1, seed=9)
    assert np.array_equal(gpu.ref_segments(R).astype(np.int64), seg)
    seq, offs = _reads(text, [0, 4000], seg, 60, 3)
    want = oracle.map_bruteforce(text, oracle.prepare_reads(seq, offs, seed=9), offs, K, "all", segments=seg)
    B = gpu.index_reads(R, seq, offs, 12, k=K)
    _same(gpu.map(R, B, "all"), want)


def test_bad_contig_lists_and_bytes_are_refused(gpu):
    for cs in ([1], [0, 0], [0, 50], [0, 30, 20]):
        with pytest.raises(gpu.PeanutError) as e:
            gpu.pack_reference(b"ACGT" * 10, contigs=cs)
        assert e.value.status == 1
    with pytest.raises(gpu.PeanutError):
        gpu.pack_reference(b"ACGTRACGT")
    with pytest.raises(gpu.PeanutError):
        gpu.pack_reference(b"ACGTACGT", gap_min=0, contigs=[0])
