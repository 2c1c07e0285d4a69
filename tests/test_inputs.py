"""The seeded input recipes of the batched and serving workloads (host only)."""
import numpy as np

import synth


def test_uneven_batches_cover_all_reads_within_bounds():
    for n, seed in ((10_000_000, 77), (3_000_000, 5), (70_000, 1)):
        b = synth.uneven_batches(n, seed)
        sizes = np.diff(b)
        assert b[0] == 0 and b[-1] == n
        assert (sizes > 0).all()
        assert (sizes[:-1] >= 1 << 16).all() and (sizes <= 1 << 21).all()
        assert synth.uneven_batches(n, seed) == b  # seeded
    # log-uniform: sizes spread over the whole range
    s = np.diff(synth.uneven_batches(200_000_000, 3))[:-1]
    assert s.min() < 1 << 17 and s.max() > 1 << 20


def test_request_stream_shape():
    a, s, m = synth.request_stream(91, 2000, 50.0, 1_000, 1_000_000)
    assert np.all(np.diff(a) > 0)
    assert abs(a[-1] / 2000 - 1 / 50.0) < 0.1 / 50.0  # mean gap 1 / rate (Poisson arrivals)
    assert s.min() >= 1_000 and s.max() <= 1_000_000
    ls = np.log(s)
    assert abs(ls.mean() - (np.log(1_000) + np.log(1_000_000)) / 2) < 0.2  # log-uniform
    assert set(m) == {"all", "best"} and 0.4 < (m == "all").mean() < 0.6
    a2, s2, m2 = synth.request_stream(91, 2000, 50.0, 1_000, 1_000_000)
    assert np.array_equal(a, a2) and np.array_equal(s, s2) and np.array_equal(m, m2)


def test_serving_read_lengths_and_budgets():
    w = synth.WORKLOADS["serve_3g1"]
    ref = synth.make_reference(200_000, 3, w["repeat_frac"], w["tandem_frac"])
    r = synth.make_reads(ref, 5000, 9, lengths=w["lengths"], rate_range=w["rate_range"])
    assert r.lengths.min() >= 75 and r.lengths.max() <= 250
    k = synth.k_of_length(r.lengths, w["k"])
    assert np.array_equal(k, (r.lengths * 5 + 99) // 100)
