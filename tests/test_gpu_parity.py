"""GPU parity: every stage of the CUDA path against the CPU oracle, through the C ABI.

Floating point plays no part in this path: every comparison is exact (bit-identical hit sets,
index arrays, distance columns).  Inputs are seeded synthetic genomes and reads (synth/).
"""
import itertools
import random

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rand_seq(rng, n, alphabet="ACGT"):
    return "".join(rng.choice(alphabet) for _ in range(n))


def concat(reads):
    offs = np.zeros(len(reads) + 1, np.uint64)
    offs[1:] = np.cumsum([len(r) for r in reads])
    seq = "".join(r.decode() if isinstance(r, bytes) else r for r in reads).encode()
    return seq, offs


def gpu_map(gpu, ref, seq, offs, q, k=None, k_permille=None, mode="all", freq_cap=0):
    R = gpu.pack_reference(ref)
    B = gpu.index_reads(R, seq, offs, q, k=k, k_permille=k_permille, freq_cap=freq_cap)
    return gpu.map(R, B, mode), B


def assert_same_hits(got, want):
    if not np.array_equal(got, want):
        g = set(map(tuple, got.tolist()))
        w = set(map(tuple, want.tolist()))
        raise AssertionError(f"hit sets differ: {len(got)} vs {len(want)}; "
                             f"missing {sorted(w - g)[:10]}, extra {sorted(g - w)[:10]}")


# ---------------------------------------------------------------- bit-vector verification kernel


def test_bitvector_exhaustive_tiny(gpu):
    pats, txts = [], []
    for lp in range(1, 5):
        for P in itertools.product("ACGT", repeat=lp):
            for T in ("ACGTACG", "TTTT", "GATTACA", "CCGGA"):
                pats.append("".join(P).encode())
                txts.append(T.encode())
    cols = gpu.bitvector_columns(pats, txts)
    for P, T, c in zip(pats, txts, cols):
        assert c.tolist() == oracle.semiglobal_column(P, T).tolist(), (P, T)


@pytest.mark.parametrize("m", [1, 2, 31, 32, 33, 63, 64, 65, 100, 127, 128, 129, 191, 192, 193, 250, 255])
def test_bitvector_word_boundaries(gpu, m):
    rng = random.Random(m)
    pats, txts = [], []
    for t in range(12):
        alpha = "ACGT" if t % 3 else "AC"
        P = rand_seq(rng, m, alpha)
        # texts that contain a mutated copy of P, and random ones
        src = list(P)
        for _ in range(rng.randint(0, 4)):
            x = rng.randrange(len(src))
            op = rng.random()
            if op < 0.5:
                src[x] = rng.choice("ACGT")
            elif op < 0.75:
                src.insert(x, rng.choice("ACGT"))
            elif len(src) > 1:
                del src[x]
        T = rand_seq(rng, rng.randint(0, 40), alpha) + "".join(src) + rand_seq(rng, rng.randint(1, 40), alpha)
        pats.append(P.encode())
        txts.append(T.encode())
    cols = gpu.bitvector_columns(pats, txts)
    for P, T, c in zip(pats, txts, cols):
        assert c.tolist() == oracle.semiglobal_column(P, T).tolist()


# ---------------------------------------------------------------- q-group index (Algorithm 1)


def _expected_index(seq, offs, q, ref=None, cap=None):
    codes, pay = oracle.canonical_text(seq, offs, q)
    if ref is not None:
        fc, _ = oracle.frequent_qgrams(ref, q, cap)
        keep = ~np.isin(codes, fc)
        codes, pay = codes[keep], pay[keep]
    return oracle.qgroup_build(codes, pay, q, 32)


@pytest.mark.parametrize("layout", ["interleaved", "sampled_s", "w64"])
@pytest.mark.parametrize("q", [4, 7, 11])
def test_index_equals_algorithm1(gpu, q, layout):
    ref = synth.make_reference(50_000, 21)
    reads = synth.make_reads(ref, 300, 5, lengths=(60, 90, 120), rate_range=(0.0, 0.03))
    R = gpu.pack_reference(ref)
    B = gpu.index_reads(R, reads.seq, reads.offsets, q, k=1, freq_cap=1 << 30, layout=layout)
    I, S, Sp, O = gpu.export_index(B)
    eI, eS, eSp, eO, d = _expected_index(reads.seq, reads.offsets, q)
    assert I.tolist() == eI.tolist()
    assert S.tolist() == eS.tolist()
    assert Sp.tolist() == eSp.tolist()
    # O: the same occurrences in every q-gram's interval (order within an interval is free)
    for x in range(d):
        a, b = int(Sp[x]), int(Sp[x + 1])
        assert sorted(O[a:b].tolist()) == sorted(eO[a:b].tolist())


def test_index_excludes_frequent_qgrams(gpu):
    ref = synth.make_reference(200_000, 22, tandem_frac=0.05)
    reads = synth.make_reads(ref, 400, 6, lengths=(100,), rate_range=(0.0, 0.02))
    q, cap = 10, 40
    R = gpu.pack_reference(ref)
    B = gpu.index_reads(R, reads.seq, reads.offsets, q, k=2, freq_cap=cap)
    I, S, Sp, O = gpu.export_index(B)
    eI, eS, eSp, eO, d = _expected_index(reads.seq, reads.offsets, q, ref, cap)
    assert I.tolist() == eI.tolist() and S.tolist() == eS.tolist() and Sp.tolist() == eSp.tolist()
    thr, lc = gpu.export_read_params(B)
    assert lc.sum() > 0  # tandem runs make some reads low-complexity


# ---------------------------------------------------------------- full hit sets


def test_hand_example(gpu):
    got, _ = gpu_map(gpu, b"TTACGTTACGATT", b"ACGTA", [0, 5], q=2, k=1)
    assert_same_hits(got, oracle.map_bruteforce(b"TTACGTTACGATT", b"ACGTA", [0, 5], 1))
    got, _ = gpu_map(gpu, b"TTACGTTACGATT", b"ACGTA", [0, 5], q=2, k=1, mode="best")
    assert got.tolist() == [(0, 1, 5, 0)]


@pytest.mark.parametrize("seed", range(6))
def test_tiny_random_vs_bruteforce(gpu, seed):
    rng = random.Random(500 + seed)
    n = rng.choice([80, 300, 2000])
    unit = rand_seq(rng, rng.randint(1, 3))
    ref = list(rand_seq(rng, n))
    for _ in range(3):
        p = rng.randrange(0, n - 40)
        for t in range(rng.randint(15, 40)):
            ref[p + t] = unit[t % len(unit)]
    ref = "".join(ref)
    reads = []
    for _ in range(40):
        m = rng.choice([16, 20, 33, 64, 65])
        p = rng.randrange(-4, n - m + 4)
        s = "".join(ref[x] if 0 <= x < n else "A" for x in range(p, p + m))
        s = list(s)
        for _ in range(rng.randint(0, 2)):
            s[rng.randrange(m)] = rng.choice("ACGT")
        s = "".join(s)
        if rng.random() < 0.5:
            s = synth.revcomp_ascii(s.encode()).tobytes().decode()
        reads.append(s)
    seq, offs = concat(reads)
    for k in (0, 1, 2):
        q = 5 if k < 2 else 4
        for mode in ("all", "best"):
            want = oracle.map_bruteforce(ref.encode(), seq, offs, k, mode)
            for cap in (0, 3):  # default and tiny cap (forces low-complexity handling)
                got, _ = gpu_map(gpu, ref.encode(), seq, offs, q, k=k, mode=mode, freq_cap=cap)
                assert_same_hits(got, want)


def test_uniform_1mbp_10k_full(gpu):
    """The small workload in full: 1 Mbp uniform reference, 10,000 reads of 100 bp, q = 11, k = 5."""
    ref, reads, w = synth.make_workload("uniform_1mbp_10k")
    want = oracle.map_filter(ref, reads.seq, reads.offsets, 5, 11)
    got, B = gpu_map(gpu, ref, reads.seq, reads.offsets, 11, k=5)
    assert_same_hits(got, want)
    assert len(got) >= 0.99 * reads.n  # planted reads are found


@pytest.mark.parametrize("mode", ["all", "best"])
def test_repeat_rich_scaled(gpu, mode):
    """Repeat families and tandem runs at 2 Mbp; q = 16, k = 5, both modes."""
    ref, reads, w = synth.make_workload("repeat_100mbp_1m", ref_len=2_000_000, n_reads=3000)
    want = oracle.map_filter(ref, reads.seq, reads.offsets, 5, 16, mode)
    for cap in (0, 16):
        got, B = gpu_map(gpu, ref, reads.seq, reads.offsets, 16, k=5, mode=mode, freq_cap=cap)
        assert_same_hits(got, want)
    thr, lc = gpu.export_read_params(B)
    assert lc.sum() > 0


def test_uneven_lengths_scaled(gpu):
    ref, reads, w = synth.make_workload("uneven_3g1_10m", ref_len=1_000_000, n_reads=3000)
    k = synth.k_of_length(reads.lengths, "5pct")
    want = oracle.map_filter(ref, reads.seq, reads.offsets, k, 12)
    got, B = gpu_map(gpu, ref, reads.seq, reads.offsets, 12, k_permille=50)
    assert_same_hits(got, want)


@pytest.mark.parametrize("q,stride", [(8, 1), (8, 2), (6, 1), (6, 3)])
def test_hit_heavy_reads_take_every_window_path(gpu, q, stride):
    """Short q on a 1 Mbp reference: ~2,800 (q = 8) and ~46,000 (q = 6) q-gram hits per read, so
    reads go through the warp, block (<= 16,384 hits) and global (radix-sorted) window paths."""
    ref, reads, w = synth.make_workload("repeat_100mbp_1m", ref_len=1_000_000, n_reads=300)
    for mode in ("all", "best"):
        want = oracle.map_filter(ref, reads.seq, reads.offsets, 5, q, mode)
        B = gpu.index_reads(gpu.pack_reference(ref), reads.seq, reads.offsets, q, k=5, stride=stride)
        got = gpu.map(B.ref, B, mode)
        assert_same_hits(got, want)
    st = gpu.get_map_stats(B)
    assert st["hits"] > reads.n * (2000 if q == 8 else 20000) / stride
    # the block path (1,025-12,288 hits per read) and the global radix-sorted path (more) ran
    if q == 8:
        assert st["med_reads"] > 0, st
    else:
        assert st["big_reads"] > 0, st


def test_candidates_cover_every_true_end(gpu):
    ref, reads, w = synth.make_workload("repeat_100mbp_1m", ref_len=500_000, n_reads=800)
    ends = oracle.map_filter(ref, reads.seq, reads.offsets, 5, 16, "ends")
    R = gpu.pack_reference(ref)
    B = gpu.index_reads(R, reads.seq, reads.offsets, 16, k=5, freq_cap=8)
    gpu.map(R, B)
    cr, cs, lo, hi = gpu.export_candidates(B)
    # candidates are sorted, disjoint and non-touching per (read, strand)
    key = cr.astype(np.int64) * 2 + cs
    order = np.lexsort((lo, key))
    assert np.array_equal(order, np.arange(order.size))
    same = key[1:] == key[:-1]
    assert np.all(lo[1:][same] > hi[:-1][same] + 1)
    cover = {}
    for r, s, a, b in zip(cr.tolist(), cs.tolist(), lo.tolist(), hi.tolist()):
        cover.setdefault((r, s), []).append((a, b))
    for r, s, e, d in ends.tolist():
        assert any(a <= e <= b for a, b in cover.get((r, s), [])), (r, s, e)


# ---------------------------------------------------------------- invariants and edge cases


def test_strand_symmetry_and_batch_invariance(gpu):
    ref, reads, w = synth.make_workload("repeat_100mbp_1m", ref_len=1_000_000, n_reads=1000)
    R = gpu.pack_reference(ref)
    full = gpu.map(R, gpu.index_reads(R, reads.seq, reads.offsets, 16, k=5))
    # the same reads split in two batches
    a = reads.slice(0, 400)
    b = reads.slice(400, reads.n)
    ha = gpu.map(R, gpu.index_reads(R, a.seq, a.offsets, 16, k=5))
    hb = gpu.map(R, gpu.index_reads(R, b.seq, b.offsets, 16, k=5))
    hb["read"] += 400
    assert_same_hits(np.concatenate([ha, hb]), full)
    # reverse-complemented reads: strands swap
    rc = np.concatenate([synth.revcomp_ascii(reads.seq[int(reads.offsets[i]):int(reads.offsets[i + 1])])
                         for i in range(reads.n)])
    hr = gpu.map(R, gpu.index_reads(R, rc, reads.offsets, 16, k=5))
    hr["strand"] ^= 1
    assert_same_hits(oracle.sort_hits(hr), full)
    # another q gives the same answer
    h12 = gpu.map(R, gpu.index_reads(R, reads.seq, reads.offsets, 12, k=5))
    assert_same_hits(h12, full)


def test_edge_cases(gpu):
    rng = random.Random(7)
    ref = rand_seq(rng, 5000)
    # reads overhanging both reference ends, a minimal-threshold read (m = q (k + 1)), a poly-A read
    reads = [("GGGG" + ref[:60]), ref[-50:] + "TTTT", ref[1000:1024], "A" * 40, ref[2000:2100]]
    seq, offs = concat(reads)
    want = oracle.map_bruteforce(ref.encode(), seq, offs, 3, "all")
    got, _ = gpu_map(gpu, ref.encode(), seq, offs, 6, k=3)
    assert_same_hits(got, want)
    # a reference containing the poly-A read many times
    ref2 = ("A" * 300 + rand_seq(rng, 200)) * 6
    want = oracle.map_bruteforce(ref2.encode(), seq, offs, 3, "all")
    for cap in (0, 4):
        got, _ = gpu_map(gpu, ref2.encode(), seq, offs, 6, k=3, freq_cap=cap)
        assert_same_hits(got, want)


def test_invalid_inputs_rejected(gpu):
    R = gpu.pack_reference(b"ACGT" * 100)
    with pytest.raises(gpu.PeanutError) as e:
        gpu.index_reads(R, b"ACGXACGTACGTACGT", [0, 16], 4, k=0)
    assert e.value.status == 1
    with pytest.raises(gpu.PeanutError) as e:  # t = 16 + 1 - 8 * 3 < 1
        gpu.index_reads(R, b"ACGTACGTACGTACGT", [0, 16], 8, k=2)
    assert e.value.status == 1
    with pytest.raises(gpu.PeanutError) as e:
        gpu.index_reads(R, b"A" * 300, [0, 300], 8, k=2)
    assert e.value.status == 1
    with pytest.raises(gpu.PeanutError) as e:
        gpu.pack_reference(b"ACGTR")
    assert e.value.status == 1
    with pytest.raises(gpu.PeanutError) as e:
        gpu.index_reads(R, b"ACGT", [0, 4], 20, k=0)
    assert e.value.status == 5


def test_no_hits_and_random_reads(gpu):
    ref = synth.make_reference(300_000, 31)
    reads = synth.make_reads(ref, 200, 9, lengths=(100,), random_frac=1.0)
    got, B = gpu_map(gpu, ref, reads.seq, reads.offsets, 16, k=5)
    assert got.size == 0
    assert gpu.get_map_stats(B)["results"] == 0


def test_device_variants_match_host(gpu):
    import torch
    ref, reads, w = synth.make_workload("uniform_1mbp_10k", n_reads=2000)
    R = gpu.pack_reference(ref)
    host = gpu.map(R, gpu.index_reads(R, reads.seq, reads.offsets, 11, k=5))
    d_seq = torch.from_numpy(reads.seq).cuda()
    d_off = torch.from_numpy(reads.offsets.astype(np.int64)).cuda()
    B = gpu.index_reads_device(R, d_seq, d_off, 11, k=5)
    dh = gpu.map_device(R, B)
    assert dh.n == len(host)
    assert_same_hits(dh.to_numpy(), host)
    gpu.use_torch_allocator()
    try:
        B2 = gpu.index_reads(R, reads.seq, reads.offsets, 11, k=5)
        assert_same_hits(gpu.map(R, B2), host)
    finally:
        gpu.use_default_allocator()


def test_objects_outlive_an_allocator_switch(gpu):
    """An object made under one device-memory provider is released by that provider even after
    another is installed, and leaves no error behind for the next call."""
    import gc
    ref, reads, w = synth.make_workload("uniform_1mbp_10k", n_reads=500)
    R = gpu.pack_reference(ref)
    want = gpu.map(R, gpu.index_reads(R, reads.seq, reads.offsets, 11, k=5))
    gpu.use_torch_allocator()
    try:
        B = gpu.index_reads(R, reads.seq, reads.offsets, 11, k=5)
        dh = gpu.map_device(R, B)
    finally:
        gpu.use_default_allocator()
    del B, dh
    gc.collect()
    assert_same_hits(gpu.map(R, gpu.index_reads(R, reads.seq, reads.offsets, 11, k=5)), want)
    assert (gpu.bitvector_columns([b"ACGT"], [b"TTACGTT"])[0].tolist()
            == oracle.semiglobal_column(b"ACGT", b"TTACGTT").tolist())


@pytest.mark.parametrize("k", [7, 20, 40])
def test_large_budgets_span_several_blocks(gpu, k):
    """Long reads with large error budgets keep several 64-bit blocks of the bit-vector column
    active at once (Myers' block cut-off starts and drops blocks along the text)."""
    rng = random.Random(900 + k)
    ref = rand_seq(rng, 3000)
    reads = []
    for _ in range(30):
        m = rng.choice([130, 192, 200, 250])
        p = rng.randrange(0, 3000 - m)
        s = list(ref[p:p + m])
        for _ in range(rng.randint(0, k)):
            x = rng.randrange(len(s))
            op = rng.random()
            if op < 0.6:
                s[x] = rng.choice("ACGT")
            elif op < 0.8:
                s.insert(x, rng.choice("ACGT"))
            elif len(s) > 2:
                del s[x]
        s = "".join(s)[:m]
        if rng.random() < 0.5:
            s = synth.revcomp_ascii(s.encode()).tobytes().decode()
        reads.append(s)
    seq, offs = concat(reads)
    q = max(1, min((len(r) + 1 - 1) // (k + 1) for r in reads))  # t = m + 1 - q (k + 1) >= 1
    for mode in ("all", "best"):
        want = oracle.map_bruteforce(ref.encode(), seq, offs, k, mode)
        got, _ = gpu_map(gpu, ref.encode(), seq, offs, q, k=k, mode=mode)
        assert_same_hits(got, want)


def test_host_array_views_equal_structured_result(gpu):
    ref, reads, w = synth.make_workload("uniform_1mbp_10k", n_reads=1500)
    R = gpu.pack_reference(ref)
    B = gpu.index_reads(R, reads.seq, reads.offsets, 11, k=5)
    want = gpu.map(R, B)
    for _ in range(2):  # the second call reuses a pooled page-locked block
        h = gpu.map_arrays(R, B)
        assert h.n == len(want)
        assert np.array_equal(h.read, want["read"]) and np.array_equal(h.strand, want["strand"])
        assert np.array_equal(h.end.astype(np.int64), want["end"]) and np.array_equal(h.dist, want["dist"])
        h.free()


@pytest.mark.parametrize("layout", ["sampled_s", "w64"])
def test_index_layouts_map_identically(gpu, layout):
    """The sampled-S and w = 64 layouts of the batch index (Section "The q-group index") give the
    oracle's hit set, at q = 16 with frequent q-grams and at q = 11, every q-gram and sampled."""
    ref, reads, w = synth.make_workload("repeat_100mbp_1m", ref_len=2_000_000, n_reads=2000)
    R = gpu.pack_reference(ref)
    for q, stride in ((16, 1), (16, 4), (11, 1)):
        want = oracle.map_filter(ref, reads.seq, reads.offsets, 5, q)
        B = gpu.index_reads(R, reads.seq, reads.offsets, q, k=5, stride=stride, layout=layout)
        assert_same_hits(gpu.map(R, B), want)
