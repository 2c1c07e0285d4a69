"""Pins for the CPU oracle: the paper's definitions, hand-worked values, brute force, invariants.

Nothing here touches the CUDA library.  Every expected value comes from a definition of the
paper (cited per test), from an independent textbook routine written here in plain Python, or
from a fixture under tests/golden/.
"""
import itertools
import os
import random
from collections import Counter, defaultdict

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
COMP = {"A": "T", "C": "G", "G": "C", "T": "A"}


def rc(s: str) -> str:
    return "".join(COMP[c] for c in reversed(s))


def levenshtein(a: str, b: str) -> int:
    """Textbook global edit distance (Wagner & Fischer 1974), unit costs."""
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[len(b)]


def semiglobal_by_substrings(P: str, R: str):
    """D[j] = min over every substring R[s..j] (including the empty one) of the global edit
    distance to P: the defining property of E[m][j] in Section "Validation"."""
    return [min(levenshtein(P, R[s:j + 1]) for s in range(0, j + 2)) for j in range(len(R))]


def canonical_from_D(D, k):
    """(end, dist) of the leftmost minimum of each maximal run of D <= k."""
    out, j = [], 0
    while j < len(D):
        if D[j] > k:
            j += 1
            continue
        e = j
        while e + 1 < len(D) and D[e + 1] <= k:
            e += 1
        run = D[j:e + 1]
        mn = min(run)
        out.append((j + run.index(mn), mn))
        j = e + 1
    return out


def read_fixture(name):
    rows = defaultdict(list)
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key].append(vals)
    return rows


def rand_seq(rng, n, alphabet="ACGT"):
    return "".join(rng.choice(alphabet) for _ in range(n))


def as_tuples(h):
    return [(int(r), int(s), int(e), int(d)) for r, s, e, d in h]


# ---------------------------------------------------------------- semiglobal DP


def test_hand_example_columns_and_tuples():
    g = read_fixture("semiglobal_hand.txt")
    ref, read, k = g["ref"][0][0], g["read"][0][0], int(g["k"][0][0])
    D0 = [int(x) for x in g["D0"][0]]
    D1 = [int(x) for x in g["D1"][0]]
    assert list(oracle.semiglobal_column(read.encode(), ref.encode())) == D0
    assert list(oracle.semiglobal_column(rc(read).encode(), ref.encode())) == D1
    want_all = [(0, int(s), int(e), int(d)) for s, e, d in g["all"]]
    want_best = [(0, int(s), int(e), int(d)) for s, e, d in g["best"]]
    offs = [0, len(read)]
    assert as_tuples(oracle.map_bruteforce(ref.encode(), read.encode(), offs, k)) == want_all
    assert as_tuples(oracle.map_bruteforce(ref.encode(), read.encode(), offs, k, "best")) == want_best
    for q in (1, 2):  # t = 6 - q(k+1) >= 1
        assert as_tuples(oracle.map_filter(ref.encode(), read.encode(), offs, k, q)) == want_all
        assert as_tuples(oracle.map_filter(ref.encode(), read.encode(), offs, k, q, "best")) == want_best


def test_semiglobal_equals_min_over_substrings():
    rng = random.Random(11)
    for _ in range(250):
        P = rand_seq(rng, rng.randint(1, 6))
        R = rand_seq(rng, rng.randint(1, 9), rng.choice(["ACGT", "AC", "A"]))
        assert list(oracle.semiglobal_column(P.encode(), R.encode())) == semiglobal_by_substrings(P, R)


def test_semiglobal_exhaustive_tiny():
    # every pattern of length <= 3 against every text of length <= 4 over {A, C} plus ACGT cases
    for lp in range(1, 4):
        for P in itertools.product("AC", repeat=lp):
            P = "".join(P)
            for lr in range(1, 5):
                for R in itertools.product("ACG", repeat=lr):
                    R = "".join(R)
                    got = list(oracle.semiglobal_column(P.encode(), R.encode()))
                    assert got == semiglobal_by_substrings(P, R), (P, R)


def test_semiglobal_special_cases():
    # exact occurrence ends with distance 0; a pattern against a disjoint alphabet costs min(m, j+1)+...
    assert oracle.semiglobal_column(b"ACGT", b"TTACGTTT")[5] == 0
    D = oracle.semiglobal_column(b"AAAA", b"CCCCCC")
    assert list(D) == [4] * 6  # every alignment mismatches or indels all 4 read bases
    # column of an empty-ish overlap: j = 0 allows at most one aligned base
    D = oracle.semiglobal_column(b"GA", b"ATTT")
    assert D[0] == 1  # insertion of G, then A matches R[0]
    with pytest.raises(ValueError):
        oracle.semiglobal_column(b"ACGN", b"ACGT")


# ---------------------------------------------------------------- brute force vs the filter


def _random_case(rng, n, nreads, m_choices, low_complexity):
    if low_complexity:
        unit = rand_seq(rng, rng.randint(1, 3))
        ref = list(rand_seq(rng, n))
        for _ in range(3):
            p = rng.randrange(0, n - 30)
            L = rng.randint(15, 30)
            for t in range(L):
                ref[p + t] = unit[t % len(unit)]
        ref = "".join(ref)
    else:
        ref = rand_seq(rng, n)
    reads = []
    for _ in range(nreads):
        m = rng.choice(m_choices)
        kind = rng.random()
        if kind < 0.7:
            p = rng.randrange(-5, n - m + 5)
            src = "".join(ref[x] if 0 <= x < n else rng.choice("ACGT") for x in range(p, p + m))
            s = list(src)
            for _ in range(rng.randint(0, 3)):
                op = rng.random()
                x = rng.randrange(len(s))
                if op < 0.6:
                    s[x] = rng.choice("ACGT")
                elif op < 0.8:
                    s.insert(x, rng.choice("ACGT"))
                elif len(s) > 2:
                    del s[x]
            s = "".join(s)[:m].ljust(m, "A")
            if rng.random() < 0.5:
                s = rc(s)
        else:
            s = rand_seq(rng, m)
        reads.append(s)
    offs = np.zeros(nreads + 1, np.int64)
    offs[1:] = np.cumsum([len(s) for s in reads])
    return ref, "".join(reads), offs


@pytest.mark.parametrize("seed", range(12))
def test_filter_equals_bruteforce(seed):
    rng = random.Random(1000 + seed)
    n = rng.choice([60, 200, 700])
    ref, seq, offs = _random_case(rng, n, 25, [12, 16, 20, 31], low_complexity=seed % 3 == 0)
    lens = np.diff(offs)
    for k in (0, 1, 2):
        qmax = min((int(m) + 1 - 1) // (k + 1) for m in lens)  # t = m + 1 - q(k+1) >= 1
        for q in sorted({1, 2, 3, qmax}):
            if q < 1 or q > qmax:
                continue
            for mode in ("all", "best", "ends"):
                bf = oracle.map_bruteforce(ref.encode(), seq.encode(), offs, k, mode)
                fl = oracle.map_filter(ref.encode(), seq.encode(), offs, k, q, mode)
                assert np.array_equal(bf, fl), (seed, k, q, mode)


def test_filter_bruteforce_per_read_budgets():
    rng = random.Random(5)
    ref, seq, offs = _random_case(rng, 400, 30, [20, 24, 40], low_complexity=True)
    k = np.array([rng.randint(0, 3) for _ in range(30)], np.int32)
    lens = np.diff(offs)
    q = int(min((lens[i]) // (k[i] + 1) for i in range(30)))
    for mode in ("all", "best"):
        assert np.array_equal(oracle.map_bruteforce(ref.encode(), seq.encode(), offs, k, mode),
                              oracle.map_filter(ref.encode(), seq.encode(), offs, k, q, mode))


def test_bruteforce_matches_independent_definition():
    """Brute force canonical tuples equal those read off the substring definition directly."""
    rng = random.Random(9)
    for _ in range(30):
        ref = rand_seq(rng, rng.randint(5, 14), rng.choice(["ACGT", "AC"]))
        read = rand_seq(rng, rng.randint(2, 5), "ACGT")
        k = rng.randint(0, 2)
        want = []
        for s, P in ((0, read), (1, rc(read))):
            for e, d in canonical_from_D(semiglobal_by_substrings(P, ref), k):
                want.append((0, s, e, d))
        got = as_tuples(oracle.map_bruteforce(ref.encode(), read.encode(), [0, len(read)], k))
        assert got == want


def test_filter_rejects_lossy_threshold():
    with pytest.raises(ValueError):
        oracle.map_filter(b"ACGTACGTAC", b"ACGTA", [0, 5], 1, q=3)  # t = 6 - 6 = 0


# ---------------------------------------------------------------- invariants on sampled reads


@pytest.fixture(scope="module")
def small_workload():
    ref = synth.make_reference(200_000, 1403, repeat_frac=0.05, tandem_frac=0.01)
    reads = synth.make_reads(ref, 400, 77, lengths=(100,), rate_range=(0.01, 0.04), random_frac=0.05)
    return ref, reads


def test_planted_reads_are_found(small_workload):
    """Section "The q-group index" (q-gram lemma): with t >= 1 no planted read with e <= k edits
    is lost; its true end lies in one of its runs."""
    ref, reads = small_workload
    k = 5
    ends = oracle.map_filter(ref, reads.seq, reads.offsets, k, 16, "ends")
    found = set(zip(ends["read"].tolist(), ends["strand"].tolist(), ends["end"].tolist()))
    n_checked = 0
    for i in range(reads.n):
        if 0 <= reads.truth_edits[i] <= k:
            n_checked += 1
            assert (i, int(reads.truth_strand[i]), int(reads.truth_end[i])) in found, i
    assert n_checked > 200


def test_strand_symmetry(small_workload):
    ref, reads = small_workload
    sub = reads.subset(range(0, 120))
    rcseq = np.concatenate([synth.revcomp_ascii(sub.seq[int(sub.offsets[i]):int(sub.offsets[i + 1])])
                            for i in range(sub.n)])
    a = oracle.map_filter(ref, sub.seq, sub.offsets, 5, 16)
    b = oracle.map_filter(ref, rcseq, sub.offsets, 5, 16)
    b["strand"] ^= 1
    assert np.array_equal(oracle.sort_hits(a), oracle.sort_hits(b))


def test_best_is_all_filtered_by_min(small_workload):
    ref, reads = small_workload
    a = oracle.map_filter(ref, reads.seq, reads.offsets, 5, 16, "all")
    b = oracle.map_filter(ref, reads.seq, reads.offsets, 5, 16, "best")
    mins = {}
    for r, d in zip(a["read"].tolist(), a["dist"].tolist()):
        mins[r] = min(mins.get(r, 99), d)
    keep = np.array([d == mins[r] for r, d in zip(a["read"].tolist(), a["dist"].tolist())], bool)
    assert np.array_equal(a[keep], b)


def test_parameter_invariance_q(small_workload):
    ref, reads = small_workload
    sub = reads.subset(range(0, 80))
    outs = [oracle.map_filter(ref, sub.seq, sub.offsets, 5, q) for q in (10, 13, 16)]
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_exact_copies_have_distance_zero():
    ref = synth.make_reference(50_000, 3)
    rng = random.Random(3)
    starts = [rng.randrange(0, 50_000 - 100) for _ in range(20)]
    reads = [ref[s:s + 100].tobytes().decode() for s in starts]
    offs = np.arange(0, 2001, 100)
    h = oracle.map_filter(ref, "".join(reads).encode(), offs, 5, 16)
    got = {(int(r), int(e)): int(d) for r, s, e, d in h if s == 0}
    for i, s in enumerate(starts):
        assert got[(i, s + 99)] == 0


def test_random_reads_do_not_map():
    ref = synth.make_reference(1_000_000, 4)
    reads = synth.make_reads(ref, 50, 12, lengths=(100,), random_frac=1.0)
    h = oracle.map_filter(ref, reads.seq, reads.offsets, 5, 16)
    assert h.size == 0


# ---------------------------------------------------------------- Algorithm 1


def test_qgroup_hand_example():
    g = read_fixture("qgroup_hand.txt")
    q, w = int(g["q"][0][0]), int(g["w"][0][0])
    codes = np.array([int(x) for x in g["codes"][0]], np.uint64)
    pos = np.array([int(x) for x in g["positions"][0]], np.uint64)
    I, S, Sp, O, d = oracle.qgroup_build(codes, pos, q, w)
    assert [format(int(x), "0%db" % w) for x in I] == g["I"][0]
    assert S.tolist() == [int(x) for x in g["S"][0]]
    assert Sp.tolist() == [int(x) for x in g["Sp"][0]]
    assert O.tolist() == [int(x) for x in g["O"][0]]
    code, a, b = (int(x) for x in g["indexpair"][0])
    assert oracle.indexpair(I, S, Sp, w, code) == (a, b)
    assert sorted(O[a:b].tolist()) == [int(x) for x in g["positions_of"][0][1:]]


@pytest.mark.parametrize("q,w", [(3, 32), (4, 4), (5, 64), (6, 32), (2, 3)])
def test_qgroup_indexpair_equals_dict(q, w):
    rng = np.random.default_rng(q * 100 + w)
    T = 500
    codes = rng.integers(0, min(4 ** q, 40), T).astype(np.uint64) * (4 ** q // 40 if 4 ** q > 40 else 1)
    codes = np.where(rng.random(T) < 0.5, codes, rng.integers(0, 4 ** q, T).astype(np.uint64))
    pay = np.arange(T, dtype=np.uint64) * 7 + 3
    I, S, Sp, O, d = oracle.qgroup_build(codes, pay, q, w)
    ref = defaultdict(list)
    for c, p in zip(codes.tolist(), pay.tolist()):
        ref[c].append(p)
    assert d == len(ref)
    assert sum(bin(int(x)).count("1") for x in I) == d
    assert int(Sp[-1]) == T
    for g in range(4 ** q):  # exhaustive over all q-grams
        a, b = oracle.indexpair(I, S, Sp, w, g)
        assert sorted(O[a:b].tolist()) == sorted(ref.get(g, [])), g


def test_index_size_closed_forms():
    g = read_fixture("index_size.txt")
    # epsilon = 1: ratio 1 + eps/(16(1+eps)) = 1 + 1/32
    q, T = 10, 4 ** 10
    ratio = oracle.qgroup_index_words(q, T) / oracle.qgram_index_words(q, T)
    assert round((ratio - 1) * 100) == int(g["eps1_disadvantage_percent"][0][0])
    # break-even K = 16/15 for K > 1: sizes equal
    K = float(g["break_even_K"][0][0])
    T = 10 ** 6
    four_q = K * T
    qg = 2 / 32 * four_q + T + T
    assert abs(qg / (four_q + T) - 1) < 1e-6
    # q = 16, |T| = 1e8
    K = 4 ** 16 / 1e8
    assert round(K, 2) == float(g["q16_T1e8_K"][0][0])
    ratio = oracle.qgroup_index_words(16, 10 ** 8) / oracle.qgram_index_words(16, 10 ** 8)
    assert round(ratio * 100 / 10) * 10 == int(g["q16_T1e8_ratio_percent"][0][0])


def test_lemma_threshold_values():
    # t = m + 1 - q(k + 1): 100 bp, k = 5 at q = 11 and q = 16
    assert oracle.lemma_threshold(100, 11, 5) == 35
    assert oracle.lemma_threshold(100, 16, 5) == 5
    assert oracle.lemma_threshold(100, 16, 6) < 1  # at most 5 errors are guaranteed at q = 16


# ---------------------------------------------------------------- helpers of the GPU design


def test_canonical_text_matches_strings():
    rng = random.Random(2)
    reads = [rand_seq(rng, rng.randint(8, 20)) for _ in range(30)]
    offs = np.zeros(31, np.int64)
    offs[1:] = np.cumsum([len(s) for s in reads])
    q = 6
    codes, pay = oracle.canonical_text("".join(reads).encode(), offs, q)
    want_c, want_p = [], []
    val = {"A": 0, "C": 1, "G": 2, "T": 3}

    def code(s):
        x = 0
        for ch in s:
            x = 4 * x + val[ch]
        return x
    for r, s in enumerate(reads):
        for i in range(len(s) - q + 1):
            g, h = code(s[i:i + q]), code(rc(s[i:i + q]))
            want_c.append(min(g, h))
            want_p.append((r << 9) | (int(g > h) << 8) | i)
    assert codes.tolist() == want_c and pay.tolist() == want_p


def test_frequent_qgrams_match_counter():
    ref = synth.make_reference(30_000, 8, tandem_frac=0.05)
    s = ref.tobytes().decode()
    q, cap = 8, 20
    cnt = Counter(min(s[p:p + q], rc(s[p:p + q])) for p in range(len(s) - q + 1))
    val = {"A": 0, "C": 1, "G": 2, "T": 3}
    want = sorted((sum(val[c] << (2 * (q - 1 - t)) for t, c in enumerate(g)), n)
                  for g, n in cnt.items() if n > cap)
    codes, counts = oracle.frequent_qgrams(ref, q, cap)
    assert list(zip(codes.tolist(), counts.tolist())) == want
    assert len(want) > 0


# ---------------------------------------------------------------- the input generator


def _splitmix_py(seed, stream, i):
    M = (1 << 64) - 1
    G = 0x9E3779B97F4A7C15

    def mix(z):
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)
    key = mix((seed * 0x100000001B3 + stream * 0x632BE59BD9B4E019 + G) & M)
    return mix((key + (i + 1) * G) & M)


def test_generator_is_splitmix64():
    got = synth.counter_u64(1403, 12, 5, 4)
    assert got.tolist() == [_splitmix_py(1403, 12, i) for i in range(5, 9)]


def test_generator_deterministic_and_acgt():
    a = synth.make_reference(100_000, 1, repeat_frac=0.3, tandem_frac=0.02)
    b = synth.make_reference(100_000, 1, repeat_frac=0.3, tandem_frac=0.02)
    assert np.array_equal(a, b)
    assert set(np.unique(a).tolist()) <= set(b"ACGT")
    ra = synth.make_reads(a, 1000, 5, lengths=(50, 75, 100, 150, 250), rate_range=(0.02, 0.02))
    rb = synth.make_reads(a, 1000, 5, lengths=(50, 75, 100, 150, 250), rate_range=(0.02, 0.02))
    assert np.array_equal(ra.seq, rb.seq) and set(np.unique(ra.lengths).tolist()) == {50, 75, 100, 150, 250}


# ---------------------------------------------------------------- postprocessing


def test_postprocess_hand_example():
    """Start, hit-rank and mapping quality of the hand example's hits, worked by hand."""
    g = read_fixture("semiglobal_hand.txt")
    ref, read, k = g["ref"][0][0], g["read"][0][0], int(g["k"][0][0])
    h = oracle.map_bruteforce(ref.encode(), read.encode(), [0, len(read)], k)
    want = [tuple(int(x) for x in row) for row in read_fixture("postprocess_hand.txt")["hit"]]
    start, rank, mapq = oracle.annotate(ref.encode(), read.encode(), [0, len(read)], h)
    got = [(int(s), int(e), int(d), int(a), int(b), int(c))
           for (_, s, e, d), a, b, c in zip(as_tuples(h), start, rank, mapq)]
    assert got == want


@pytest.mark.parametrize("seed", range(3))
def test_start_is_leftmost_substring_at_the_hit_distance(seed):
    """The start equals the smallest i with Levenshtein(pattern, R[i..end]) = dist, found by trying
    every substring with the textbook distance (independent of the oracle's backward DP)."""
    rng = random.Random(40 + seed)
    ref = rand_seq(rng, 300, "ACGT" if seed else "AC")
    reads = []
    for _ in range(12):
        m = rng.randint(5, 14)
        p = rng.randrange(0, 300 - m)
        s = list(ref[p:p + m])
        for _ in range(rng.randint(0, 2)):
            x = rng.randrange(len(s))
            op = rng.random()
            if op < 0.5:
                s[x] = rng.choice("ACGT")
            elif op < 0.75:
                s.insert(x, rng.choice("ACGT"))
            elif len(s) > 3:
                del s[x]
        reads.append("".join(s))
    seq = "".join(reads).encode()
    offs = np.concatenate([[0], np.cumsum([len(r) for r in reads])])
    h = oracle.map_bruteforce(ref.encode(), seq, offs, 2)
    assert len(h) > 10
    start, rank, mapq = oracle.annotate(ref.encode(), seq, offs, h)
    for (r, s, e, d), st in zip(as_tuples(h), start.tolist()):
        P = reads[r] if s == 0 else rc(reads[r])
        dists = [levenshtein(P, ref[i:e + 1]) for i in range(0, e + 2)]
        assert min(dists) == d
        assert st == dists.index(d)


def test_rank_counts_hits_at_least_as_good_and_mapq_special_cases():
    """Hit-rank = the read's hits with distance <= the hit's (counted here directly); quality 255
    at rank 1 (the hand example) and exactly 10 x when (rank - 1) / |P| = 10^-x."""
    rng = random.Random(5)
    unit = "ACGTTGCA"
    ref = (unit * 125)  # 1,000 bases: a 100-base read maps at every period
    read = (unit * 13)[:100]
    h = oracle.map_bruteforce(ref.encode(), read.encode(), [0, 100], 3)
    start, rank, mapq = oracle.annotate(ref.encode(), read.encode(), [0, 100], h)
    d = h["dist"]
    for x in range(len(h)):
        assert rank[x] == int((d <= d[x]).sum())
    n = len(ref)
    for x in range(len(h)):
        if rank[x] == 1:
            assert mapq[x] == 255
        elif rank[x] - 1 == n // 10:  # (rank - 1) / |P| = 10^-1
            assert mapq[x] == 10
    # 11 separate exact copies of a read on a 100-base reference (no G, so its reverse complement
    # GGTT never occurs): rank 11, -10 log10(10 / 100) = 10 exactly
    ref2 = "AACCTT" * 11 + "T" * 34
    h2 = oracle.map_bruteforce(ref2.encode(), b"AACC", [0, 4], 0)
    assert len(h2) == 11
    s2, r2, q2 = oracle.annotate(ref2.encode(), b"AACC", [0, 4], h2)
    assert r2.tolist() == [11] * 11 and q2.tolist() == [10] * 11
    assert s2.tolist() == [6 * x for x in range(11)]
