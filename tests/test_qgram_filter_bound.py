"""The bound behind the q'-gram filter on candidate ranges, checked by brute force on the CPU.

Claim (the q-gram lemma of Section "The q-group index", applied at one end position): if the
semiglobal distance D[j] of a read of length m ending at text position j is at most k, then at
least T' = m - q' + 1 - q' k text positions p in [j - m - k + 1, j - q' + 1] start a q'-gram that
also occurs in the read, and since the intact q'-grams are a sub-multiset of the read's, this
stays true after discounting, for any q'-gram, the window's occurrences beyond the read's count.
The GPU filter drops an end only when such a count over whole 16-base blocks around the window
(with the discount for the read's four most frequent q'-grams) is below T', so the claim is what
makes it exact.  Here D comes from
the oracle's DP (Section "Validation") and the count is written out plainly; the inputs include
tandem runs, reads overhanging the text start, and budgets up to the largest T' >= 1 allows.
"""
import random
from collections import Counter

import numpy as np
import pytest

import oracle

QF = 4


def qgrams(s: str, q: int) -> set:
    return {s[i:i + q] for i in range(len(s) - q + 1)}


def window_count(text: str, read_set: set, j: int, m: int, k: int, q: int) -> int:
    lo, hi = max(0, j - m - k + 1), j - q + 1
    return sum(1 for p in range(lo, hi + 1) if text[p:p + q] in read_set)


def block_bound(text: str, read_set: set, j: int, m: int, k: int, q: int) -> int:
    """The GPU's count for the 16-base block of ends holding j: every q'-gram start in blocks
    J - D .. J, D = ceil((m + k - 1) / 16), J = j // 16 (q'-grams running past the text end
    count as absent here; the GPU may count them, which only raises its bound)."""
    J = j // 16
    D = (m + k - 1 + 15) // 16
    lo = max(0, (J - D) * 16)
    hi = min(J * 16 + 15, len(text) - q)
    return sum(1 for p in range(lo, hi + 1) if text[p:p + q] in read_set)


def tracked_block_bound(text: str, read: str, j: int, m: int, k: int, q: int, tracked: int = 4) -> int:
    """The GPU's tighter count: the block count above less, for the read's `tracked` most frequent
    q'-grams (ties to the smaller code), how far their count in those blocks exceeds their count
    in the read (the intact q'-grams are a sub-multiset of the read's)."""
    cnt_read = Counter(read[i:i + q] for i in range(len(read) - q + 1))
    code = lambda g: int("".join("ACGT".index(c).__str__() for c in g), 4)
    top = sorted(cnt_read, key=lambda g: (-cnt_read[g], code(g)))[:tracked]
    J = j // 16
    D = (m + k - 1 + 15) // 16
    lo = max(0, (J - D) * 16)
    hi = min(J * 16 + 15, len(text) - q)
    grams = [text[p:p + q] for p in range(lo, hi + 1)]
    in_read = sum(1 for g in grams if g in cnt_read)
    cnt_u = Counter(grams)
    return in_read - sum(max(0, cnt_u[g] - cnt_read[g]) for g in top)


def mutate(rng, s, edits):
    s = list(s)
    for _ in range(edits):
        x = rng.randrange(len(s))
        op = rng.random()
        if op < 0.6:
            s[x] = rng.choice("ACGT")
        elif op < 0.8:
            s.insert(x, rng.choice("ACGT"))
        elif len(s) > 2:
            del s[x]
    return "".join(s)


def cases(seed, n):
    rng = random.Random(seed)
    for _ in range(n):
        m = rng.choice([12, 20, 33, 50, 64, 100])
        k = rng.randint(0, max(0, (m - QF) // QF - 1))  # T' >= 1
        unit = "".join(rng.choice("ACGT") for _ in range(rng.randint(1, 4)))
        if rng.random() < 0.4:  # tandem-rich text and read
            text = "".join(unit[i % len(unit)] if rng.random() < 0.9 else rng.choice("ACGT")
                           for i in range(rng.randint(m, 4 * m)))
        else:
            text = "".join(rng.choice("ACGT") for _ in range(rng.randint(m, 4 * m)))
        p = rng.randrange(-5, len(text) - m + 5)
        src = "".join(text[x] if 0 <= x < len(text) else rng.choice("ACGT") for x in range(p, p + m))
        read = mutate(rng, src, rng.randint(0, k + 1))[:m] if len(src) else src
        if len(read) < QF:
            continue
        yield read, text, k


@pytest.mark.parametrize("seed", range(4))
def test_every_end_within_k_keeps_t_prime_qgrams(seed):
    checked = 0
    for read, text, k in cases(seed, 150):
        m = len(read)
        T = m - QF + 1 - QF * k
        assert T >= 1
        D = oracle.semiglobal_column(read.encode(), text.encode())
        rs = qgrams(read, QF)
        for j in np.flatnonzero(D <= k).tolist():
            c = window_count(text, rs, j, m, k, QF)
            assert c >= T, (read, text, j, int(D[j]), c, T)
            assert block_bound(text, rs, j, m, k, QF) >= c
            assert tracked_block_bound(text, read, j, m, k, QF) >= T, (read, text, j)
            checked += 1
    assert checked > 500


def test_bound_is_tight_enough_to_reject_unrelated_text():
    """On random text a random 100 bp read's window count stays far below T' (k = 5): the
    filter removes windows that hold no alignment."""
    rng = random.Random(9)
    read = "".join(rng.choice("ACGT") for _ in range(100))
    text = "".join(rng.choice("ACGT") for _ in range(3000))
    rs = qgrams(read, QF)
    T = 100 - QF + 1 - QF * 5
    counts = [block_bound(text, rs, j, 100, 5, QF) for j in range(200, 3000, 16)]
    assert max(counts) < T


def test_tracked_discount_rejects_a_partly_tandem_read_inside_a_long_run():
    """A read whose last 30 bases are (AC)^15 against the interior of a 120-base AC run: every
    window position holds ACAC or CACA, both in the read, so the plain count passes, but the read
    holds each only ~14 times and the discounted count falls far below T'."""
    rng = random.Random(3)
    read = "".join(rng.choice("ACGT") for _ in range(70)) + "AC" * 15
    text = "".join(rng.choice("ACGT") for _ in range(300)) + "AC" * 60 + "".join(rng.choice("ACGT") for _ in range(300))
    m, k = 100, 5
    T = m - QF + 1 - QF * k
    rs = qgrams(read, QF)
    j = 300 + 110  # an end deep inside the run
    assert block_bound(text, rs, j, m, k, QF) >= T
    assert tracked_block_bound(text, read, j, m, k, QF) < T
