"""GPU parity on the low-complexity paths that only very repetitive references reach.

A (read, strand) whose frequent q-grams have more than 12,288 occurrence clusters (plus counting
ranges) is too large for the block merge and goes to the warp k-way merge; one with 32 or more
cluster lists (distinct frequent (q-gram, orientation) pairs) is merged by one lane.  On the
3.1 Gbp workload these segments are the tandem-run reads.  Here a 7 Mbp reference carries
13,000 poly-A and 13,000 poly-T runs (20-30 bp, so A^16 has ~260,000 occurrences in 26,000
clusters) and 300 identical copies of a 300 bp family (every 16-gram of it occurs 300 times, in
300 clusters), so that reads overlapping a run take the k-way merge and reads from the family
take the one-lane merge.  Hit sets are compared element by element with the oracle (q-gram
filter + windowed DP, Sections "Filtration" and "Validation") in both modes, and the path
counters of the map call must show that both branches ran.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

K, Q = 5, 16
RUN_SLOT = 220          # one poly run per slot of the run region
N_RUNS = 26_000         # half poly-A, half poly-T
FAMILY_LEN, FAMILY_COPIES = 300, 300


def _reference():
    rng = np.random.default_rng(1403)
    run_region = N_RUNS * RUN_SLOT
    fam_region = FAMILY_COPIES * 600
    tail = 1_000_000
    n = run_region + fam_region + tail
    ref = synth.make_reference(n, 77)
    runs = []
    for x in range(N_RUNS):
        length = int(rng.integers(20, 31))
        start = x * RUN_SLOT + int(rng.integers(70, RUN_SLOT - length - 70))
        ref[start:start + length] = ord("A") if x % 2 == 0 else ord("T")
        runs.append((start, length))
    family = ref[n - 1000:n - 1000 + FAMILY_LEN].copy()  # a piece of the unique tail
    fam_starts = []
    for c in range(FAMILY_COPIES):
        st = run_region + c * 600 + int(rng.integers(100, 200))
        ref[st:st + FAMILY_LEN] = family
        fam_starts.append(st)
    return ref, runs, fam_starts, run_region + fam_region


def _mutate(rng, read, n_sub):
    r = read.copy()
    for _ in range(n_sub):
        x = int(rng.integers(0, r.size))
        r[x] = np.frombuffer(b"ACGT", np.uint8)[(("ACGT".index(chr(r[x])) + int(rng.integers(1, 4))) % 4)]
    return r


@pytest.fixture(scope="module")
def lowcx_case(gpu):
    ref, runs, fam_starts, tail0 = _reference()
    rng = np.random.default_rng(5)
    reads = []
    # ordinary reads from the unique tail
    tail = synth.make_reads(ref[tail0:], 120, 31, lengths=(100,), rate_range=(0.0, 0.03))
    reads += [np.frombuffer(tail.read(i), np.uint8) for i in range(tail.n)]
    # reads overlapping a poly run by 18-30 bases at either end of the read
    for x in rng.choice(len(runs), 30, replace=False):
        st, ln = runs[int(x)]
        ov = int(rng.integers(18, ln + 1))
        # the read ends with the run's first ov bases, or starts with its last ov bases
        a = st + ov - 100 if rng.random() < 0.5 else st + ln - ov
        reads.append(_mutate(rng, ref[a:a + 100], int(rng.integers(0, 3))))
    # reads from the family (all of their q-grams are frequent)
    for x in rng.choice(len(fam_starts), 10, replace=False):
        st = fam_starts[int(x)] + int(rng.integers(0, FAMILY_LEN - 100))
        reads.append(_mutate(rng, ref[st:st + 100], int(rng.integers(0, 3))))
    # one pure poly-A read and one poly-A read with two substitutions
    reads.append(np.full(100, ord("A"), np.uint8))
    reads.append(_mutate(rng, np.full(100, ord("A"), np.uint8), 2))
    offs = np.zeros(len(reads) + 1, np.uint64)
    offs[1:] = np.cumsum([r.size for r in reads])
    seq = np.concatenate(reads)
    R = gpu.pack_reference(ref)
    # the oracle's hit sets, both modes computed side by side (ctypes releases the GIL)
    with ThreadPoolExecutor(2) as ex:
        want = dict(zip(("all", "best"), ex.map(lambda m: oracle.map_filter(ref, seq, offs, K, Q, m),
                                                ("all", "best"))))
    return ref, seq, offs, R, want


@pytest.mark.parametrize("mode", ["all", "best"])
@pytest.mark.parametrize("stride", [1, 4])
def test_kmerge_and_serial_merge_equal_oracle(gpu, lowcx_case, mode, stride):
    ref, seq, offs, R, wants = lowcx_case
    want = wants[mode]
    B = gpu.index_reads(R, seq, offs, Q, k=K, stride=stride)
    got = gpu.map(R, B, mode)
    st = gpu.get_map_stats(B)
    if not np.array_equal(got, want):
        g, w = set(map(tuple, got.tolist())), set(map(tuple, want.tolist()))
        raise AssertionError(f"{len(got)} vs {len(want)}: missing {sorted(w - g)[:8]}, extra {sorted(g - w)[:8]}")
    assert len(want) > 3000  # the family reads map to ~300 copies each
    assert st["lowcx_reads"] >= 30, st
    if stride == 1:  # (sampling every 4th q-gram leaves fewer cluster lists than either path needs)
        assert st["lowcx_rest_segments"] > st["lowcx_serial_segments"] > 0, st  # warp k-way and one-lane merges
    B.free()
