"""Pins of the oracle's unknown-base and multi-contig rules, on the CPU.

Section "The q-group index" (encoding paragraph): N becomes a random base and long runs of N stay
out of the index; Section "Overview": every step runs per chromosome.  The readings (a seeded
counter-based generator for the random bases; runs of at least gap_min Ns and contig boundaries
cut the reference into segments that no alignment leaves) are pinned here against things other
than the oracle itself: the generators' published outputs, hand-built segment lists, and the
single-contig oracle (pinned in test_oracle.py) run on each segment's own text.
"""
import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "generators.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def test_generators_match_published_outputs():
    rows = _golden()
    assert len(rows) == 6
    for row in rows:
        if row[0] == "splitmix64":
            assert oracle.splitmix64(int(row[1]), int(row[2])) == int(row[3], 16), row
        else:
            s = b"" if row[1] == "-" else row[1].encode()
            assert oracle.fnv1a64(s) == int(row[2], 16), row


def _rand(rng, n):
    return "".join(rng.choice("ACGT") for _ in range(n))


def test_segments_of_hand_built_references():
    # contigs [0, 10), [10, 40), [40, 50); a 6-N gap inside contig 1 (gap_min 5), a 4-N run that
    # stays (shorter than gap_min), a gap at the start of contig 2, an N run crossing the 1 | 2
    # boundary (split by it: 3 Ns end contig 1, 5 Ns start contig 2)
    seq = ("ACGTACGTAC"                                 # contig 0: 0..9
           + "ACGTA" + "NNNNNN" + "CGTA" + "NNNN" + "ACGTACGT" + "NNN"  # contig 1: 10..39
           + "NNNNN" + "ACGTA")                         # contig 2: 40..49
    assert len(seq) == 50
    text, seg = oracle.prepare_reference(seq.encode(), [0, 10, 40], gap_min=5, seed=7)
    assert seg.tolist() == [[0, 10], [10, 15], [21, 40], [45, 50]]
    # a contig that is one whole gap has no segment; gap_min 1 turns every N into a gap
    _, seg = oracle.prepare_reference(b"ACGTNNNNNACG", [0, 4, 9], gap_min=3)
    assert seg.tolist() == [[0, 4], [9, 12]]
    _, seg = oracle.prepare_reference(b"ACNGT", [0], gap_min=1)
    assert seg.tolist() == [[0, 2], [3, 5]]


def test_unknown_bases_take_the_generators_top_bits_and_case_folds():
    seq = b"acgtNNnnACGT" + b"N" * 30
    for seed in (0, 1, 2 ** 63 + 5):
        text, _ = oracle.prepare_reference(seq, [0], gap_min=16, seed=seed)
        t = bytes(text).decode()
        assert t[:4] == "ACGT" and t[8:12] == "ACGT"
        for p, c in enumerate(seq.decode()):
            if c in "Nn":
                assert t[p] == "ACGT"[oracle.splitmix64(seed, p + 1) >> 62], (seed, p)
    # seed 0, position 0 is output 1 of the generator: e220... -> top bits 11 -> T
    assert bytes(oracle.prepare_reference(b"N", [0], seed=0)[0]) == b"T"


def test_replacement_bases_are_uniform():
    n = 40_000
    text, _ = oracle.prepare_reference(b"N" * n, [0], gap_min=n + 1, seed=1706)
    counts = np.bincount(np.frombuffer(bytes(text), np.uint8), minlength=256)[[65, 67, 71, 84]]
    chi2 = float(((counts - n / 4) ** 2 / (n / 4)).sum())
    assert chi2 < 16.3, counts  # 3 degrees of freedom, p = 0.001


def test_bad_bytes_and_contig_lists_are_refused():
    for seq, cs in ((b"ACGX", [0]), (b"ACGT", [1]), (b"ACGT", [0, 0]), (b"ACGT", [0, 4]), (b"ACGT", [0, 3, 2])):
        with pytest.raises(ValueError):
            oracle.prepare_reference(seq, cs)
    with pytest.raises(ValueError):
        oracle.prepare_reads(b"ACGTR", [0, 5])


def test_read_replacement_depends_on_the_read_alone():
    rng = random.Random(4)
    r1 = "ACGTNNACGTTTGCANGT"
    r2 = _rand(rng, 30)
    batch_a = (r1 + r2).encode()
    batch_b = (r2 + r1.lower()).encode()
    a = bytes(oracle.prepare_reads(batch_a, [0, len(r1), len(r1) + len(r2)], seed=11)).decode()
    b = bytes(oracle.prepare_reads(batch_b, [0, len(r2), len(r1) + len(r2)], seed=11)).decode()
    assert a[:len(r1)] == b[len(r2):]
    assert a[len(r1):] == r2
    h = oracle.fnv1a64(r1.encode())
    for i, c in enumerate(r1):
        if c == "N":
            assert a[i] == "ACGT"[oracle.splitmix64(11 ^ h, i + 1) >> 62]
        else:
            assert a[i] == c


def _shift(h, d):
    h = h.copy()
    h["end"] += d
    return h


def _union(parts):
    return oracle.sort_hits(np.concatenate(parts))


def _reads_over(rng, text, n, m, k, anchors):
    """Reads of length m from the text with up to k substitutions, many straddling `anchors`."""
    reads = []
    for x in range(n):
        if x % 2 == 0 and anchors:
            a = rng.choice(anchors)
            p = max(0, min(len(text) - m, a - rng.randrange(1, m)))
        else:
            p = rng.randrange(0, len(text) - m + 1)
        r = list(text[p:p + m])
        for _ in range(rng.randint(0, k)):
            i = rng.randrange(m)
            r[i] = rng.choice("ACGT")
        reads.append("".join(r))
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum([len(r) for r in reads])
    return "".join(reads).encode(), offs


def _best(h):
    """Best stratum of a hit set in (read, strand, end) order."""
    if h.size == 0:
        return h
    keep = np.zeros(h.size, bool)
    for r in np.unique(h["read"]):
        sel = h["read"] == r
        keep |= sel & (h["dist"] == h["dist"][sel].min())
    return h[keep]


@pytest.mark.parametrize("seed", range(3))
def test_segmented_map_is_the_union_of_per_segment_maps(seed):
    """Mapping against contigs (and gaps) equals mapping every segment's own text with the
    single-contig definition, shifted to its start; the filter route gives the same set."""
    rng = random.Random(seed)
    parts = [_rand(rng, rng.randint(120, 260)) for _ in range(3)]
    # contig 1 repeats the end of contig 0 so that reads straddling the boundary have a true
    # in-contig copy too; contig 2 is preceded by a 20-N gap inside contig 1
    parts[1] = parts[0][-40:] + parts[1]
    seq = parts[0] + parts[1] + "N" * 20 + parts[2]
    c1 = len(parts[0])
    text, seg = oracle.prepare_reference(seq.encode(), [0, c1], gap_min=16, seed=seed)
    g0 = c1 + len(parts[1])
    assert seg.tolist() == [[0, c1], [c1, g0], [g0 + 20, len(seq)]]
    m, k, q = 30, 2, 6
    reads, offs = _reads_over(rng, bytes(text).decode(), 40, m, k, [c1, g0, g0 + 20])
    want_ends = _union([_shift(oracle.map_bruteforce(text[a:b], reads, offs, k, "ends"), a) for a, b in seg])
    got_ends = oracle.map_bruteforce(text, reads, offs, k, "ends", segments=seg)
    assert np.array_equal(got_ends, want_ends)
    want = _union([_shift(oracle.map_bruteforce(text[a:b], reads, offs, k, "all"), a) for a, b in seg])
    got = oracle.map_bruteforce(text, reads, offs, k, "all", segments=seg)
    assert np.array_equal(got, want)
    assert np.array_equal(oracle.map_filter(text, reads, offs, k, q, "all", segments=seg), want)
    assert np.array_equal(oracle.map_filter(text, reads, offs, k, q, "best", segments=seg), _best(want))
    # the segments matter: straddling reads find ends the whole-text map has and the segmented
    # one does not
    whole = oracle.map_bruteforce(text, reads, offs, k, "ends")
    assert whole.size > got_ends.size


def test_annotation_stays_inside_the_segment():
    rng = random.Random(8)
    a, b = _rand(rng, 150), _rand(rng, 150)
    seq = a + b
    text, seg = oracle.prepare_reference(seq.encode(), [0, 150])
    # a read whose best alignment in contig 1 starts at its first base, and whose 6 leading
    # bases also match the end of contig 0
    read = a[-6:] + b[:34]
    reads, offs = read.encode(), np.array([0, 40])
    hits = oracle.map_bruteforce(text, reads, offs, 6, "all", segments=seg)
    st, rank, mapq = oracle.annotate(text, reads, offs, hits, segments=seg)
    assert np.all(st >= np.where(hits["end"] >= 150, 150, 0))
    # each hit's start equals the one the single-contig oracle gives on its segment's own text
    for x, h in enumerate(hits):
        sa, sb = (0, 150) if h["end"] < 150 else (150, 300)
        one = oracle.map_bruteforce(text[sa:sb], reads, offs, 6, "all")
        y = np.flatnonzero((one["end"] == h["end"] - sa) & (one["strand"] == h["strand"]))
        assert y.size == 1
        s1, _, _ = oracle.annotate(text[sa:sb], reads, offs, one)
        assert st[x] == s1[y[0]] + sa
    assert any(st[hits["end"] >= 150] == 150)
