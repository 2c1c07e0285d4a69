"""Pins of the oracle's mate pairing (Section "Postprocessing", paired-end mode), on the CPU:
a hit list worked by hand, and simulated fragments whose true pair must come out with the
fragment's length as its span, whatever the strand the fragment lies on."""
import os
import random

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pairs_hand.txt")


def _hand():
    params, hits, pairs = {}, [], {"all": [], "best": []}
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "params":
            params = dict(zip(f[1::2], f[2::2]))
        elif f[0] == "hit":
            hits.append(tuple(int(v) for v in f[1:]))
        else:
            pairs[f[1]].append(tuple(int(v) for v in f[2:]))
    return params, hits, pairs


def test_hand_example():
    params, hits, pairs = _hand()
    h = np.empty(len(hits), oracle.HIT_DTYPE)
    h["read"] = [x[1] for x in hits]
    h["strand"] = [x[2] for x in hits]
    h["end"] = [x[3] for x in hits]
    h["dist"] = [x[4] for x in hits]
    starts = np.array([x[5] for x in hits])
    lens = [int(v) for v in params["lengths"].split(",")]
    offs = np.concatenate([[0], np.cumsum(lens)])
    cs = [int(v) for v in params["contigs"].split(",")]
    for mode in ("all", "best"):
        got = oracle.pair_hits(h, starts, offs, int(params["n"]), int(params["min_insert"]),
                               int(params["max_insert"]), mode, cs)
        assert [tuple(int(v) for v in row) for row in got.tolist()] == pairs[mode], mode


def _revcomp(s):
    return s[::-1].translate(str.maketrans("ACGT", "TGCA"))


@pytest.mark.parametrize("seed", range(3))
def test_simulated_fragments_pair_with_their_length(seed):
    rng = random.Random(seed)
    ref = "".join(rng.choice("ACGT") for _ in range(3000))
    mates, truth = [], []
    for f in range(12):
        L = rng.randint(200, 400)
        p = rng.randrange(0, 3000 - L)
        frag = ref[p:p + L]
        m1, m2 = rng.randint(30, 50), rng.randint(30, 50)
        a, b = frag[:m1], _revcomp(frag[-m2:])
        if f % 2:  # the fragment read from the other strand: mate 1 is the reverse one
            a, b = _revcomp(frag[-m1:]), frag[:m2]
        mates += [a, b]
        truth.append((p, p + L - 1, L))
    seq = "".join(mates).encode()
    offs = np.concatenate([[0], np.cumsum([len(m) for m in mates])])
    hits = oracle.map_bruteforce(ref.encode(), seq, offs, 2, "all")
    starts, _, _ = oracle.annotate(ref.encode(), seq, offs, hits)
    pairs = oracle.pair_hits(hits, starts, offs, len(ref), 150, 450, "all")
    for f, (a, b, L) in enumerate(truth):
        sel = hits["read"][pairs["i1"]] // 2 == f
        spans = {(int(starts[i1] if hits["strand"][i1] == 0 else starts[i2]),
                  int(hits["end"][i2] if hits["strand"][i1] == 0 else hits["end"][i1]))
                 for i1, i2 in zip(pairs["i1"][sel], pairs["i2"][sel])}
        assert (a, b) in spans, f
        best = oracle.pair_hits(hits, starts, offs, len(ref), 150, 450, "best")
        sb = best[hits["read"][best["i1"]] // 2 == f]
        assert sb.size >= 1 and np.all(sb["score"] == 2 * (len(mates[2 * f]) * len(mates[2 * f + 1])))
    # every reported pair obeys the definition
    for i1, i2 in zip(pairs["i1"], pairs["i2"]):
        assert hits["read"][i1] % 2 == 0 and hits["read"][i2] == hits["read"][i1] + 1
        assert hits["strand"][i1] != hits["strand"][i2]
        fwd, rev = (i1, i2) if hits["strand"][i1] == 0 else (i2, i1)
        assert 150 <= hits["end"][rev] - starts[fwd] + 1 <= 450


def test_bad_input_is_refused():
    h = np.zeros(2, oracle.HIT_DTYPE)
    h["read"] = [1, 0]  # not grouped by read
    with pytest.raises(ValueError):
        oracle.pair_hits(h, [0, 0], [0, 10, 20], 100, 10, 20)
    with pytest.raises(ValueError):  # odd number of reads
        oracle.pair_hits(h[:0], [], [0, 10, 20, 30], 100, 10, 20)
    with pytest.raises(ValueError):
        oracle.pair_hits(h[:0], [], [0, 10, 20], 100, 30, 20)
