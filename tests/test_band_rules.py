"""The rules the GPU alignment kernels rest on, checked on the CPU against the oracle's alignment
(Section "Postprocessing": the actual alignment of each hit).

The kernels for hits of distance d <= 7 fill only the diagonals lo <= c - i <= lo + d, with
Delta = n - m and lo = ceil((Delta - d) / 2): a path of cost d that visits offset c - i = delta pays
at least |delta| + |Delta - delta| for its gaps, so no path of cost d leaves that band.  Rows whose
band lies inside the rectangle (1 <= c <= n) take a cell's value from its diagonal neighbour a alone
(a, or a + 1 when the bases differ and neither the left nor the up neighbour is below a, since
diagonal steps never lower the value and neighbours differ by at most one); the other rows take the
minimum of the three moves.  Each cell keeps only its traceback direction (the diagonal when it is
optimal, else the reference-only step, else the read-only step) and the walk back reads those
alone.  The model below restates exactly those rules in plain Python, and its alignment must equal
the oracle's full-matrix one on every random pair, including pairs over two letters (many ties),
lengths that differ by the whole distance, and patterns of one base.
"""
import random

import pytest

import oracle

INF = 0xFFFF


def _distance(p, t):
    """Edit distance of p and t, both ends fixed (the full matrix, row by row)."""
    prev = list(range(len(t) + 1))
    for i in range(1, len(p) + 1):
        cur = [i] + [0] * len(t)
        for c in range(1, len(t) + 1):
            cur[c] = min(prev[c - 1] + (p[i - 1] != t[c - 1]), prev[c] + 1, cur[c - 1] + 1)
        prev = cur
    return prev[-1]


def _band_cigar(p, t, d):
    """The kernels' alignment of p against t at distance d, as an extended CIGAR string."""
    m, n = len(p), len(t)
    assert abs(n - m) <= d
    w, lo = d + 1, -((d - (n - m)) // 2)
    row = [lo + o if 0 <= lo + o <= n else INF for o in range(w)]
    dirs = [[1] * w]  # row 0: reference-only steps
    for i in range(1, m + 1):
        drow = [0] * w
        if i + lo >= 1 and i + lo + w - 1 <= n:  # the unit-step rule
            for o in range(w):
                a = row[o]
                lf = row[o - 1] if o > 0 else INF  # already row i
                up = row[o + 1] if o + 1 < w else INF  # still row i - 1
                mis = p[i - 1] != t[i + lo + o - 1]
                ge = lf >= a and up >= a
                drow[o] = 0 if not mis else (3 if ge else (1 if lf < a else 2))
                row[o] = a + (1 if mis and ge else 0)
        else:  # the minimum of the three moves
            for o in range(w):
                c = i + lo + o
                v, dr = INF, 0
                if 0 <= c <= n:
                    if c == 0:
                        v, dr = i, 2
                    else:
                        mis = int(p[i - 1] != t[c - 1])
                        dg = row[o] + mis
                        lf = row[o - 1] + 1 if o > 0 else INF
                        up = row[o + 1] + 1 if o + 1 < w else INF
                        v = min(dg, lf, up)
                        dr = 3 * mis if dg == v else (1 if lf == v else 2)
                row[o], drow[o] = v, dr
        dirs.append(drow)
    assert row[n - m - lo] == d
    ops, i, c = [], m, n
    while i > 0 or c > 0:
        o = c - i - lo
        assert 0 <= o < w, "the walk back left the band"
        dr = dirs[i][o]
        if dr in (0, 3):
            ops.append("=" if dr == 0 else "X")
            i, c = i - 1, c - 1
        elif dr == 1:
            ops.append("D")
            c -= 1
        else:
            ops.append("I")
            i -= 1
    ops.reverse()
    out, k = [], 0
    while k < len(ops):
        e = k
        while e < len(ops) and ops[e] == ops[k]:
            e += 1
        out.append(f"{e - k}{ops[k]}")
        k = e
    return "".join(out)


def _mutate(rng, s, edits, alphabet):
    s = list(s)
    for _ in range(edits):
        op = rng.random()
        y = rng.randrange(len(s) + 1)
        if op < 0.4 and y < len(s):
            s[y] = rng.choice(alphabet)
        elif op < 0.7 or len(s) <= 1:
            s.insert(y, rng.choice(alphabet))
        elif y < len(s):
            del s[y]
    return "".join(s)


@pytest.mark.parametrize("alphabet", ["ACGT", "AC"])
def test_band_rules_give_the_oracles_alignment(alphabet):
    rng = random.Random(1403 + len(alphabet))
    seen = set()
    for _ in range(2500):
        m = rng.choice([1, 2, 3, rng.randint(4, 12), rng.randint(13, 40)])
        p = "".join(rng.choice(alphabet) for _ in range(m))
        t = _mutate(rng, p, rng.randint(0, 9), alphabet)
        if not t:
            continue
        d = _distance(p, t)
        if d > 7:
            continue
        assert _band_cigar(p, t, d) == oracle.cigar(p.encode(), t.encode(), d), (p, t, d)
        seen.add((d, len(t) - len(p)))
    # every distance, and lengths that differ by the whole distance either way
    assert {x for x, _ in seen} == set(range(8))
    assert any(dl == x > 0 for x, dl in seen) and any(dl == -x < 0 for x, dl in seen)


def test_band_is_never_wider_than_the_distance_plus_one():
    for d in range(8):
        for delta in range(-d, d + 1):
            lo = -((d - delta) // 2)
            hi = (delta + d) // 2
            assert lo <= 0 <= hi and lo <= delta <= hi and hi - lo <= d
            # every offset in the band can be visited by some path of cost d, and the two
            # offsets just outside cannot
            for off in (lo, hi):
                assert abs(off) + abs(delta - off) <= d
            for off in (lo - 1, hi + 1):
                assert abs(off) + abs(delta - off) > d
