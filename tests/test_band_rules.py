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


# ---- the alignment start of a hit (the backward pass of Section "Validation") ----------------
#
# The start kernel takes a hit of distance d <= 7 ending at j through the reversed pattern against
# the reference read leftwards from j, column c = 1 .. min(m + d, j + 1 - segment start), and needs
# only E(m, c) for c in [m - d, m + d]; every path of cost <= d to those cells stays within
# |c - i| <= d, so it keeps the 2d + 1 cells of that band, one per diagonal, as 2-bit fields of one
# word (cell k: row c - d + k; the upper bit of each field a spacer that lets the carry of the
# addition below cross into the next cell).  Cells above row 0 take the virtual value c - i (as
# row 0 takes c), which satisfies the recurrence whatever the bases, so the band needs no edge
# cases.  Per column: D(k) = 1 exactly when the cell exceeds its diagonal neighbour, which by the
# unit-step rule is (bases differ) and not (the left neighbour is below it) and not (the cell above
# in this column is below it); the last condition chains down the column and is solved for all
# cells at once by one addition (Z(k) = G(k) | (P(k) & Z(k - 1)) is the carry vector of
# (G | P) + G).  The vertical differences of the column then follow from the previous column's and
# D; the value of row m comes from the tracked top cell and popcounts.


def _u(x):
    return x & 0xFFFFFFFF


def _start_model(pat, ref, j, d, sa):
    """The start kernel's rules restated: the leftmost start of the hit, or None (not a hit)."""
    m = len(pat)
    rev = pat[::-1]  # row i <-> rev[i - 1]
    C = min(m + d, j + 1 - sa)
    W = 2 * d + 1
    E = sum(1 << (2 * k) for k in range(W))  # the cells' value bits
    ODD = E << 1  # the spacers
    UP = sum(1 << (2 * k) for k in range(d + 1, W))  # column 0: E(i, 0) = |i|
    UN = sum(1 << (2 * k) for k in range(1, d + 1))
    v0 = d  # the top cell's value
    base = lambda i: rev[i - 1] if 1 <= i <= m else 0  # any base outside the pattern
    pw = 0  # the band's pattern bases, cell k at bits 2k
    for k in range(W):
        pw |= base(k - d) << (2 * k)
    score0 = m
    best = 0 if score0 == d else -1
    ok = True
    for c in range(1, C + 1):
        pw = (pw >> 2) | (base(c + d) << (2 * (W - 1)))
        t = ref[j - c + 1]
        x = pw ^ (t * 0x55555555)
        mis = (x | (x >> 1)) & E
        G = (~mis & E) | ((UN >> 2) & E)
        X = G | UP | ODD
        Y = G
        Z = ((_u(X + Y) ^ X ^ Y) >> 2) & E
        D = ~Z & E
        D1 = (D << 2) & E  # D(k - 1) at cell k
        same = ~(D ^ D1) & E
        U0 = ~(UP | UN) & E
        UP, UN = ((UP & same) | (U0 & D & ~D1)) & E & ~1, ((UN & same) | (U0 & ~D & D1)) & E & ~1
        v0 += D & 1
        k = m - c + d  # row m's cell
        if 0 <= k < W:
            low = ((1 << (2 * k + 1)) - 1) & E
            val = v0 + bin(UP & low).count("1") - bin(UN & low).count("1")
            if val == d:
                best = c
            if val < d:
                ok = False
    if best < 0 or not ok:
        return None
    return j - best + 1


_CODE = {"A": 0, "C": 1, "G": 2, "T": 3}


@pytest.mark.parametrize("alphabet", ["ACGT", "AC"])
def test_start_rules_give_the_oracles_starts(alphabet):
    import numpy as np
    rng = random.Random(1706 + len(alphabet))
    checked = set()
    for trial in range(60):
        n = rng.randint(40, 160)
        ref = "".join(rng.choice(alphabet) for _ in range(n))
        contigs = [0] if trial % 3 else [0, rng.randint(10, n - 10)]
        text, seg = oracle.prepare_reference(ref.encode(), contigs, gap_min=16)
        text = bytes(text).decode()
        reads = []
        for _ in range(6):
            m = rng.randint(1, 30)
            p = rng.randrange(0, n - m + 1)
            reads.append(_mutate(rng, text[p:p + m], rng.randint(0, 4), alphabet) or "A")
        offs = np.concatenate([[0], np.cumsum([len(r) for r in reads])]).astype(np.int64)
        seq = "".join(reads).encode()
        k = rng.randint(0, 7)
        hits = oracle.map_bruteforce(text.encode(), seq, offs, k, "all", segments=seg)
        if hits.size == 0:
            continue
        starts, _, _ = oracle.annotate(text.encode(), seq, offs, hits, segments=seg)
        codes = [_CODE[b] for b in text]
        for h, st in zip(hits, starts):
            read = reads[int(h["read"])]
            pat = [_CODE[b] for b in read]
            if h["strand"]:
                pat = [3 - b for b in pat[::-1]]
            j, d = int(h["end"]), int(h["dist"])
            sa = int(seg[np.searchsorted(seg[:, 1], j, side="right"), 0])
            assert _start_model(pat, codes, j, d, sa) == int(st), (read, int(h["strand"]), j, d, sa)
            checked.add(d)
            if d < 7:  # a distance above the true one is refused (some column scores below it)
                assert _start_model(pat, codes, j, d + 1, sa) is None
    assert checked >= set(range(6))
