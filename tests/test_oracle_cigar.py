"""Pins of the oracle's alignment of a hit (Section "Postprocessing": the actual alignment of
each hit), on the CPU: the hand-worked alignments of the hand example, and on random hits the
definition itself: the operations consume the whole pattern and exactly the hit's reference
bases, '=' and 'X' sit on equal and different bases, and the edits number the hit's distance."""
import os
import random
import re

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fixture(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        f = line.split()
        if f and not f[0].startswith("#"):
            rows.setdefault(f[0], []).append(f[1:])
    return rows


def test_hand_example():
    g = _fixture("semiglobal_hand.txt")
    ref, read, k = g["ref"][0][0], g["read"][0][0], int(g["k"][0][0])
    h = oracle.map_bruteforce(ref.encode(), read.encode(), [0, len(read)], k)
    st, _, _ = oracle.annotate(ref.encode(), read.encode(), [0, len(read)], h)
    got = [(int(x["strand"]), int(x["end"]), int(x["dist"]), int(s), c)
           for x, s, c in zip(h, st, oracle.alignments(ref.encode(), read.encode(), [0, len(read)], h, st))]
    want = [(int(a), int(b), int(c), int(d), e) for a, b, c, d, e in _fixture("cigar_hand.txt")["hit"]]
    assert got == want


def _check(pattern: str, text: str, d: int, cig: str):
    ops = [(int(n), o) for n, o in re.findall(r"(\d+)([=XID])", cig)]
    assert "".join(f"{n}{o}" for n, o in ops) == cig
    assert all(ops[x][1] != ops[x + 1][1] for x in range(len(ops) - 1))  # runs are maximal
    i = c = edits = 0
    for n, o in ops:
        for _ in range(n):
            if o in "=X":
                assert (pattern[i] == text[c]) == (o == "="), (pattern, text, cig)
                edits += o == "X"
                i += 1
                c += 1
            elif o == "I":
                i += 1
                edits += 1
            else:
                c += 1
                edits += 1
    assert (i, c) == (len(pattern), len(text)) and edits == d, (pattern, text, d, cig)


def test_random_hits_follow_the_definition():
    rng = random.Random(11)
    checked = 0
    for t in range(40):
        ref = "".join(rng.choice("ACGT" if t % 3 else "AC") for _ in range(400))
        reads = []
        for _ in range(6):
            m = rng.randint(8, 30)
            p = rng.randrange(0, 400 - m)
            s = list(ref[p:p + m])
            for _ in range(rng.randint(0, 3)):
                x = rng.randrange(len(s))
                op = rng.random()
                if op < 0.5:
                    s[x] = rng.choice("ACGT")
                elif op < 0.75:
                    s.insert(x, rng.choice("ACGT"))
                elif len(s) > 4:
                    del s[x]
            reads.append("".join(s))
        offs = np.concatenate([[0], np.cumsum([len(r) for r in reads])])
        seq = "".join(reads).encode()
        h = oracle.map_bruteforce(ref.encode(), seq, offs, 3, "all")
        st, _, _ = oracle.annotate(ref.encode(), seq, offs, h)
        cig = oracle.alignments(ref.encode(), seq, offs, h, st)
        for x, s, c in zip(h, st, cig):
            r = reads[int(x["read"])]
            pat = r[::-1].translate(str.maketrans("ACGT", "TGCA")) if x["strand"] else r
            _check(pat, ref[int(s):int(x["end"]) + 1], int(x["dist"]), c)
            checked += 1
    assert checked > 150


def test_a_wrong_distance_is_refused():
    try:
        oracle.cigar(b"ACGT", b"ACGA", 0)
    except ValueError:
        return
    raise AssertionError("distance 0 for ACGT / ACGA accepted")
