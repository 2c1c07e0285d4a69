"""GPU parity of paired-end mate pairing (Section "Postprocessing": mates are paired, and the
percent identities of properly paired hits are summed to form strata) against the oracle.

Fragments of 250-500 bases from a repeat-rich reference of three contigs (some straddle a contig
boundary and may not pair), read from both ends (forward-reverse, half of them with mate 1 on the
reverse strand) with sequencing errors.  The whole chain runs on the GPU (map, alignment starts,
pairing) and every step is compared element by element with the oracle's own chain: the hit
list, the starts, and the pairs with their scores, ranks and qualities, in both modes.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

K, Q = 5, 16
MIN_INS, MAX_INS = 200, 600


def _revcomp(a):
    lut = np.zeros(256, np.uint8)
    for x, y in zip(b"ACGT", b"TGCA"):
        lut[x] = y
    return lut[a[::-1]]


def _mutate(rng, r, n):
    r = r.copy()
    for _ in range(n):
        r[int(rng.integers(0, r.size))] = np.frombuffer(b"ACGT", np.uint8)[int(rng.integers(0, 4))]
    return r


def _paired(seed, n_frag, lens=(100,)):
    rng = np.random.default_rng(seed)
    ref = synth.make_reference(1_500_000, seed, repeat_frac=0.15, tandem_frac=0.01).copy()
    contigs = [0, 600_000, 1_100_000]
    # a 3 kb family copied into every contig, some copies with a few substitutions, so that
    # fragments from it pair several times with different summed identities
    fam = ref[100_000:103_000].copy()
    for c in (300_000, 700_000, 800_000, 1_200_000, 1_300_000):
        ref[c:c + 3000] = _mutate(rng, fam, int(rng.integers(0, 4)) * 3)
    mates = []
    for f in range(n_frag):
        L = int(rng.integers(250, 501))
        if f % 10 == 0:  # straddle a contig boundary
            p = contigs[1 + f % 2] - int(rng.integers(50, L - 50))
        elif f % 10 == 5:  # from the family
            p = 100_000 + int(rng.integers(0, 3000 - L))
        else:
            p = int(rng.integers(0, ref.size - L))
        frag = ref[p:p + L]
        m1, m2 = int(rng.choice(lens)), int(rng.choice(lens))
        a, b = frag[:m1], _revcomp(frag[-m2:])
        if f % 2:
            a, b = _revcomp(frag[-m1:]), frag[:m2]
        mates += [_mutate(rng, a, int(rng.integers(0, 3))), _mutate(rng, b, int(rng.integers(0, 3)))]
    offs = np.zeros(len(mates) + 1, np.int64)
    offs[1:] = np.cumsum([m.size for m in mates])
    return ref, contigs, np.concatenate(mates), offs


@pytest.fixture(scope="module")
def case(gpu):
    ref, contigs, seq, offs = _paired(7, 1500, lens=(100, 120, 150))
    R = gpu.pack_reference(ref, contigs=contigs)
    _, seg = oracle.prepare_reference(ref, contigs)  # no alignment spans two contigs
    want = {}
    for mode in ("all", "best"):
        h = oracle.map_filter(ref, seq, offs, K, Q, mode, segments=seg)  # the stratum the pairs come from
        st, _, _ = oracle.annotate(ref, seq, offs, h, segments=seg)
        want[mode] = h, st, {pm: oracle.pair_hits(h, st, offs, ref.size, MIN_INS, MAX_INS, pm, contigs)
                             for pm in ("all", "best")}
    return ref, contigs, seq, offs, R, want


@pytest.mark.parametrize("hmode", ["all", "best"])
@pytest.mark.parametrize("pmode", ["all", "best"])
def test_pairs_equal_oracle(gpu, case, hmode, pmode):
    ref, contigs, seq, offs, R, want = case
    wh, wst, wp = want[hmode]
    B = gpu.index_reads(R, seq, offs, Q, k=K)
    dh = gpu.map_device(R, B, hmode)
    assert np.array_equal(dh.to_numpy(), wh)
    start, _, _ = gpu.annotate_hits(R, B, dh)
    assert np.array_equal(start.cpu().numpy(), wst)
    got = gpu.pair_hits(R, B, dh, start, MIN_INS, MAX_INS, pmode)
    w = wp[pmode]
    for f in ("i1", "i2", "score", "rank", "mapq"):
        assert np.array_equal(got[f].astype(np.int64), w[f].astype(np.int64)), f
    if hmode == "all":
        assert got.size > 1000 and got["rank"].max() >= 4  # the family gives fragments several pairs
    B.free()


def test_pairing_edge_cases(gpu, case):
    ref, contigs, seq, offs, R, want = case
    # an odd number of reads is refused; an empty hit list gives no pairs
    B = gpu.index_reads(R, seq, offs[:4], Q, k=K)
    dh = gpu.map_device(R, B, "all")
    start, _, _ = gpu.annotate_hits(R, B, dh)
    with pytest.raises(gpu.PeanutError):
        gpu.pair_hits(R, B, dh, start, MIN_INS, MAX_INS)
    B.free()
    rnd = synth.make_reference(400, 99)  # two random 200 bp mates: no hits
    B = gpu.index_reads(R, rnd, [0, 200, 400], Q, k=K)
    dh = gpu.map_device(R, B, "all")
    start, _, _ = gpu.annotate_hits(R, B, dh)
    assert dh.n == 0 and gpu.pair_hits(R, B, dh, start, MIN_INS, MAX_INS).size == 0
    with pytest.raises(gpu.PeanutError):
        gpu.pair_hits(R, B, dh, start, 300, 200)
    B.free()
