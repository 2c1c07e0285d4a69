"""GPU postprocessing (peanut_annotate_hits) against the oracle: every hit's alignment start
(backward pass, Section "Validation"), hit-rank and mapping quality (Section "Postprocessing"),
element by element, in both modes, on the hand example, on repeat-rich references (many hits
per read, both strands, reads at the reference ends, tandem runs) and on reads of uneven length
(1 to 4 words per bit-vector column)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _kvec(offs, k=None, k_permille=None):
    lens = np.diff(np.asarray(offs, np.int64))
    return np.full(lens.size, k) if k is not None else (lens * k_permille + 999) // 1000


def _check(gpu, R, ref, seq, offs, q, mode, **kw):
    B = gpu.index_reads(R, seq, offs, q, **kw)
    dh = gpu.map_device(R, B, mode)
    h = dh.to_numpy()
    # the oracle annotates its own hit list, which the GPU's must equal first
    want = oracle.map_filter(ref, seq, offs, _kvec(offs, kw.get("k"), kw.get("k_permille")), q, mode)
    assert np.array_equal(h, want)
    start, rank, mapq = gpu.annotate_hits(R, B, dh)
    ws, wr, wq = oracle.annotate(ref, seq, offs, want)
    assert np.array_equal(start.cpu().numpy(), ws)
    assert np.array_equal(rank.cpu().numpy().astype(np.uint32), wr)
    assert np.array_equal(mapq.cpu().numpy().astype(np.int32), wq)
    return h, ws, wr


def test_hand_example(gpu):
    R = gpu.pack_reference(b"TTACGTTACGATT")
    for mode in ("all", "best"):
        h, ws, wr = _check(gpu, R, b"TTACGTTACGATT", b"ACGTA", [0, 5], 2, mode, k=1)
    assert ws.tolist() == [1] and wr.tolist() == [1]  # best stratum: the exact reverse-complement hit


@pytest.mark.parametrize("mode", ["all", "best"])
def test_repeat_rich_reads(gpu, mode):
    ref, reads, w = synth.make_workload("repeat_100mbp_1m", ref_len=1_000_000, n_reads=2000)
    R = gpu.pack_reference(ref)
    h, ws, wr = _check(gpu, R, ref, reads.seq, reads.offsets, 16, mode, k=5)
    assert len(h) > 1500 and wr.max() > 1


def test_uneven_lengths_and_budgets(gpu):
    ref, reads, w = synth.make_workload("uneven_3g1_10m", ref_len=500_000, n_reads=1500)
    R = gpu.pack_reference(ref)
    h, ws, wr = _check(gpu, R, ref, reads.seq, reads.offsets, 12, "all", k_permille=50)
    assert np.unique(reads.lengths[h["read"]]).size == 5
