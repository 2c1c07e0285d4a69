"""The bound behind the q'-gram filter on candidate ranges, checked by brute force on the CPU.

Claim (the q-gram lemma of Section "The q-group index", applied at one end position): if the
semiglobal distance D[j] of a read of length m ending at text position j is at most k, then at
least T' = m - q' + 1 - q' k text positions p in [j - m - k + 1, j - q' + 1] start a q'-gram that
also occurs in the read.  The GPU filter drops an end only when a larger count (whole 16-base
blocks around that window) is below T', so the claim is what makes it exact.  Here D comes from
the oracle's DP (Section "Validation") and the count is written out plainly; the inputs include
tandem runs, reads overhanging the text start, and budgets up to the largest T' >= 1 allows.
"""
import random

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
