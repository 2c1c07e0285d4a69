"""The reference-side q-group index (peanut_index_reference + peanut_params.ref_index = 1; the
reference index of Section "Filtration", without masking): looking the batch's q-grams up in the
reference's own index instead of streaming the reference must give exactly the streaming scan's
hits (the same number of q-gram hits, the same candidates) and the oracle's hit set, in both modes,
at every q, stride and read-length mix."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def both_scans(gpu, R, seq, offs, q, mode="all", **kw):
    out = []
    for ri in (False, True):
        B = gpu.index_reads(R, seq, offs, q, ref_index=ri, **kw)
        out.append((gpu.map(R, B, mode), gpu.get_map_stats(B)))
        B.free()
    return out


def test_hand_example(gpu):
    R = gpu.pack_reference(b"TTACGTTACGATT")
    gpu.index_reference(R, 2)
    (a, _), (b, _) = both_scans(gpu, R, b"ACGTA", [0, 5], 2, k=1)
    want = oracle.map_bruteforce(b"TTACGTTACGATT", b"ACGTA", [0, 5], 1)
    assert np.array_equal(a, want) and np.array_equal(b, want)


@pytest.mark.parametrize("mode", ["all", "best"])
def test_repeat_rich_equals_streaming_and_oracle(gpu, mode):
    ref, reads, w = synth.make_workload("repeat_100mbp_1m", ref_len=2_000_000, n_reads=3000)
    R = gpu.pack_reference(ref)
    gpu.index_reference(R, 16)
    want = oracle.map_filter(ref, reads.seq, reads.offsets, 5, 16, mode)
    for stride in (1, 4):
        (a, sa), (b, sb) = both_scans(gpu, R, reads.seq, reads.offsets, 16, mode, k=5, stride=stride)
        assert sa["hits"] == sb["hits"] and sa["candidates"] == sb["candidates"]
        assert np.array_equal(a, want) and np.array_equal(b, want)
    assert sa["lowcx_reads"] > 0


def test_uniform_and_uneven(gpu):
    ref, reads, w = synth.make_workload("uniform_1mbp_10k", n_reads=3000)
    R = gpu.pack_reference(ref)
    gpu.index_reference(R, 11)
    gpu.index_reference(R, 11)  # a second build at the same q is a no-op
    (a, _), (b, _) = both_scans(gpu, R, reads.seq, reads.offsets, 11, k=5)
    assert np.array_equal(a, b) and np.array_equal(b, oracle.map_filter(ref, reads.seq, reads.offsets, 5, 11))
    ref2, reads2, w2 = synth.make_workload("uneven_3g1_10m", ref_len=1_000_000, n_reads=2000)
    R2 = gpu.pack_reference(ref2)
    gpu.index_reference(R2, 12)
    (a, _), (b, _) = both_scans(gpu, R2, reads2.seq, reads2.offsets, 12, k_permille=50)
    k = synth.k_of_length(reads2.lengths, "5pct")
    assert np.array_equal(a, b) and np.array_equal(b, oracle.map_filter(ref2, reads2.seq, reads2.offsets, k, 12))


def test_missing_index_is_refused(gpu):
    R = gpu.pack_reference(b"ACGTTGCA" * 50)
    with pytest.raises(gpu.PeanutError) as e:
        gpu.index_reads(R, b"ACGTTGCAACGT", [0, 12], 4, k=0, ref_index=True)
    assert e.value.status == 1
