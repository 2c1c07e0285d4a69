"""The batched and served path (peanut_engine_*) and q-gram sampling against the oracle and the
plain per-batch path.

Reads of uneven length (50-250 bp, k = ceil(0.05 L)) in uneven submissions: every submission's
result must equal the oracle's hit set for it, equal the plain path's (one peanut_index_reads +
peanut_map over the submission with the one q all its reads admit), and be the same whether the
submission is mapped alone or in a mix with others, under any launch size, memory budget,
executor count, autotuned setting or sampling stride.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

LENGTHS = (50, 75, 100, 150, 250)


def k_of(m):
    return (m * 50 + 999) // 1000


@pytest.fixture(scope="module")
def world(gpu):
    ref = synth.make_reference(3_000_000, 71, 0.05, 0.01)
    reads = synth.make_reads(ref, 6000, 73, lengths=LENGTHS, rate_range=(0.0, 0.04), random_frac=0.05)
    R = gpu.pack_reference(ref)
    # uneven submissions
    bounds = [0, 1, 37, 800, 1900, 4100, 6000]
    subs = [reads.slice(a, b) for a, b in zip(bounds[:-1], bounds[1:])]
    return ref, R, subs


def plain(gpu, R, sub, mode):
    q = min(min(m // (k_of(m) + 1), 16) for m in sub.lengths)
    B = gpu.index_reads(R, sub.seq, sub.offsets, q, k_permille=50)
    try:
        return gpu.map(R, B, mode)
    finally:
        B.free()


def oracle_hits(ref, sub, mode):
    q = min(min(m // (k_of(m) + 1), 16) for m in sub.lengths)
    return oracle.map_filter(ref, sub.seq, sub.offsets, [k_of(int(m)) for m in sub.lengths], q, mode)


@pytest.fixture(scope="module")
def expected(world, gpu):
    ref, R, subs = world
    out = {}
    for i, sub in enumerate(subs):
        for mode in ("all", "best"):
            want = oracle_hits(ref, sub, mode)
            assert np.array_equal(plain(gpu, R, sub, mode), want), (i, mode)
            out[i, mode] = want
    return out


def run_engine(gpu, R, subs, modes, **kw):
    E = gpu.Engine(R, k_permille=50, **kw)
    try:
        tickets = [E.submit(s.seq, s.offsets, m) for s, m in zip(subs, modes)]
        res = [E.wait(t) for t in tickets]
        return res, E.stats()
    finally:
        E.free()


@pytest.mark.parametrize("kw", [
    dict(executors=1, autotune=False),
    dict(executors=2, autotune=False, max_reads=700),
    dict(executors=4, autotune=True),
    dict(executors=2, autotune=False, hbm_budget=3 << 30),
    dict(executors=2, autotune=False, fixed_q=12),
])
def test_engine_mix_equals_oracle(gpu, world, expected, kw):
    ref, R, subs = world
    modes = ["all", "best", "all", "best", "all", "best"]
    res, st = run_engine(gpu, R, subs, modes, **kw)
    for i, (got, m) in enumerate(zip(res, modes)):
        assert np.array_equal(got, expected[i, m]), (kw, i, m)
    assert st["completed"] == len(subs)
    assert st["reads"] >= sum(s.n for s in subs)


def test_engine_alone_equals_in_mix(gpu, world, expected):
    ref, R, subs = world
    E = gpu.Engine(R, k_permille=50, executors=2, max_reads=1500)
    try:
        alone = []
        for s in subs:
            alone.append(E.wait(E.submit(s.seq, s.offsets, "all")))
        # the same submissions interleaved with others in both modes
        t = []
        for s in subs:
            t.append((E.submit(s.seq, s.offsets, "best"), "best"))
            t.append((E.submit(s.seq, s.offsets, "all"), "all"))
        mixed = [(E.wait(x), m) for x, m in t]
    finally:
        E.free()
    for i, s in enumerate(subs):
        assert np.array_equal(alone[i], expected[i, "all"])
        assert np.array_equal(mixed[2 * i][0], expected[i, "best"])
        assert np.array_equal(mixed[2 * i + 1][0], alone[i])


def test_engine_device_submission(gpu, world, expected):
    import torch
    ref, R, subs = world
    E = gpu.Engine(R, k_permille=50, executors=2)
    try:
        t = []
        for i, s in enumerate(subs):
            d_seq = torch.from_numpy(s.seq.copy()).cuda()
            d_off = torch.from_numpy(s.offsets.astype(np.int64)).cuda()
            torch.cuda.synchronize()
            t.append((i, E.submit_device(d_seq, d_off, "all")))
        for i, x in t:
            assert np.array_equal(E.wait(x), expected[i, "all"]), i
    finally:
        E.free()


def test_engine_device_results(gpu, world, expected):
    """Results left on the device, taken after the engine is gone; a host wait on such a ticket
    copies it down; a device wait on a host-result ticket is refused."""
    import torch
    ref, R, subs = world
    E = gpu.Engine(R, k_permille=50, executors=2)
    keep = []
    try:
        d = []
        for s in subs:
            ds = torch.from_numpy(s.seq.copy()).cuda()
            do = torch.from_numpy(s.offsets.astype(np.int64)).cuda()
            d.append((ds, do))
        torch.cuda.synchronize()
        t_dev = [E.submit_device(ds, do, m, result_on_device=True) for (ds, do), m in zip(d, ("all", "best") * 3)]
        t_host = E.submit_device(d[3][0], d[3][1], "best", result_on_device=True)
        t_plain = E.submit(subs[2].seq, subs[2].offsets, "all")
        with pytest.raises(gpu.PeanutError, match="RESULT_ON_DEVICE"):
            E.wait_device(t_plain)
        assert np.array_equal(E.wait(t_plain), expected[2, "all"])
        keep = [E.wait_device(t) for t in t_dev]
        assert np.array_equal(E.wait(t_host), expected[3, "best"])
    finally:
        E.free()
    for i, (h, m) in enumerate(zip(keep, ("all", "best") * 3)):
        assert np.array_equal(h.to_numpy(), expected[i, m]), (i, m)
        h.free()


def test_engine_concurrent_clients(gpu, world, expected):
    """Eight host threads submit and wait at the same time; every result is its own."""
    import threading
    ref, R, subs = world
    E = gpu.Engine(R, k_permille=50, executors=3, max_reads=900)
    errors, got = [], {}

    def client(c):
        try:
            for rep in range(3):
                i = (c + rep) % len(subs)
                m = ("all", "best")[(c + rep) % 2]
                t = E.submit(subs[i].seq, subs[i].offsets, m)
                got[c, rep] = (i, m, E.wait(t))
        except Exception as e:  # surfaced below
            errors.append(repr(e))

    th = [threading.Thread(target=client, args=(c,)) for c in range(8)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    E.free()
    assert not errors, errors
    assert len(got) == 24
    for (c, rep), (i, m, h) in got.items():
        assert np.array_equal(h, expected[i, m]), (c, rep)


def test_engine_release_with_work_in_flight(gpu, world, expected):
    """Releasing an engine with submissions queued, running or unclaimed neither hangs nor
    leaks into a later engine."""
    ref, R, subs = world
    for executors in (1, 2):
        E = gpu.Engine(R, k_permille=50, executors=executors, max_reads=300)
        for s in subs:
            E.submit(s.seq, s.offsets, "all")
        E.submit(subs[1].seq, subs[1].offsets, "best")
        E.free()
    E = gpu.Engine(R, k_permille=50, executors=2)
    try:
        assert np.array_equal(E.wait(E.submit(subs[4].seq, subs[4].offsets, "best")), expected[4, "best"])
        assert E.wait(E.submit(subs[0].seq, subs[0].offsets, "all"), timeout_ms=60000) is not None
        # a wait that times out keeps the ticket; the next wait returns the result
        t = E.submit(subs[5].seq, subs[5].offsets, "all")
        h = E.wait(t, timeout_ms=0)
        if h is None:
            h = E.wait(t)
        assert np.array_equal(h, expected[5, "all"])
    finally:
        E.free()


def test_engine_bad_submission_fails_alone(gpu, world, expected):
    ref, R, subs = world
    bad_seq = subs[2].seq.copy()
    bad_seq[5] = ord("X")
    E = gpu.Engine(R, k_permille=50, executors=2)
    try:
        t0 = E.submit(subs[1].seq, subs[1].offsets, "all")
        tb = E.submit(bad_seq, subs[2].offsets, "all")
        t2 = E.submit(subs[3].seq, subs[3].offsets, "all")
        with pytest.raises(gpu.PeanutError, match="A/C/G/T"):
            E.wait(tb)
        assert np.array_equal(E.wait(t0), expected[1, "all"])
        assert np.array_equal(E.wait(t2), expected[3, "all"])
        too_long = np.frombuffer(b"A" * 300, np.uint8)
        tl = E.submit(too_long, np.array([0, 300], np.uint64), "all")
        with pytest.raises(gpu.PeanutError, match="lengths"):
            E.wait(tl)
        with pytest.raises(gpu.PeanutError, match="unknown ticket"):
            E.wait(10 ** 9)
    finally:
        E.free()


def test_engine_autotune_records(gpu, world, expected):
    ref, R, subs = world
    res, st = run_engine(gpu, R, subs, ["all"] * len(subs), executors=2, autotune=True)
    for i, got in enumerate(res):
        assert np.array_equal(got, expected[i, "all"])
    classes = {c["q_class"]: c for c in st["classes"]}
    # 50 bp -> 12, 75 bp -> 15, 100/150/250 bp -> 16
    assert set(classes) == {12, 15, 16}
    for c in classes.values():
        assert c["tune_candidates"] >= 1 and c["q"] in (c["q_class"], c["q_class"] - 1)
        assert 1 <= c["stride"] <= c["q"] and c["launches"] >= 1
    assert st["graph_segments"] == 0  # plain launches unless the engine asks for graphs


@pytest.mark.parametrize("executors", [1, 2])
def test_engine_graphs_equal_oracle(gpu, world, expected, executors):
    """An engine created with graphs = 1 runs each launch's sync-free stretches (the scan, binning
    and short-read windows, the filter and verification count pass, the write pass) as CUDA
    graphs; every submission's hits still equal the oracle's, in both modes, with autotuning."""
    ref, R, subs = world
    modes = ["all", "best"] * 3
    res, st = run_engine(gpu, R, subs, modes[:len(subs)], executors=executors, autotune=True, graphs=True)
    for i, (got, m) in enumerate(zip(res, modes)):
        assert np.array_equal(got, expected[i, m]), (i, m)
    assert st["graph_segments"] >= 3 * st["map_runs"] > 0


@pytest.mark.parametrize("stride", [2, 3, 4])
def test_sampling_stride_exact(gpu, stride):
    """Indexing every stride-th read q-gram with the matching threshold keeps the output exact."""
    ref = synth.make_reference(1_500_000, 81, 0.05, 0.01)
    reads = synth.make_reads(ref, 1500, 83, lengths=(150, 250), rate_range=(0.0, 0.04), random_frac=0.05)
    R = gpu.pack_reference(ref)
    ks = [k_of(int(m)) for m in reads.lengths]
    q = 13 if stride < 4 else 12
    for mode in ("all", "best"):
        want = oracle.map_filter(ref, reads.seq, reads.offsets, ks, q, mode)
        B = gpu.index_reads(R, reads.seq, reads.offsets, q, k_permille=50, stride=stride)
        got = gpu.map(R, B, mode)
        assert np.array_equal(got, want), (stride, mode)
        thr, lc = gpu.export_read_params(B)
        assert thr.min() >= 1


@pytest.mark.parametrize("q,stride,lengths", [(16, 16, (100,)), (16, 8, (100, 150)), (12, 12, (50,)),
                                               (16, 16, (150, 250)), (15, 15, (75,))])
def test_disjoint_qgram_strides_exact(gpu, q, stride, lengths):
    """Strides up to q (disjoint q-grams: each edit touches at most one, threshold = sampled - k)
    on a repeat-rich reference with tandem runs (low-complexity reads included)."""
    ref = synth.make_reference(2_000_000, 91, 0.05, 0.01)
    reads = synth.make_reads(ref, 2500, 93, lengths=lengths, rate_range=(0.0, 0.04), random_frac=0.05)
    R = gpu.pack_reference(ref)
    ks = [k_of(int(m)) for m in reads.lengths]
    for mode in ("all", "best"):
        want = oracle.map_filter(ref, reads.seq, reads.offsets, ks, min(q, 12 if 50 in lengths else q), mode)
        for cap in (0, 16):
            B = gpu.index_reads(R, reads.seq, reads.offsets, q, k_permille=50, stride=stride, freq_cap=cap)
            got = gpu.map(R, B, mode)
            assert np.array_equal(got, want), (q, stride, lengths, mode, cap)
            thr, lc = gpu.export_read_params(B)
            assert thr.min() >= 1
            if cap:
                assert lc.sum() > 0  # a small cap makes low-complexity reads


def test_sampling_thresholds_follow_the_bound(gpu):
    """On a uniform reference (no frequent q-grams) every read's threshold is the sampled-offset
    bound ceil(nq/s) - k ceil(q/s) (the q-gram lemma for s = 1)."""
    ref = synth.uniform_reference(1_000_000, 17)
    R = gpu.pack_reference(ref)
    for q, s, lengths in ((15, 1, (75, 100, 150, 250)), (15, 3, (75, 100, 150, 250)), (16, 4, (100, 150, 250)),
                          (16, 16, (100, 150, 250)), (12, 12, (50,))):
        reads = synth.make_reads(ref, 3000, 19, lengths=lengths, rate_range=(0.0, 0.04))
        L = reads.lengths.astype(np.int64)
        k = (L * 50 + 999) // 1000
        B = gpu.index_reads(R, reads.seq, reads.offsets, q, k_permille=50, stride=s)
        thr, lc = gpu.export_read_params(B)
        nq = L - q + 1
        want = -(-nq // s) - np.minimum(-(-nq // s), k * -(-q // s))
        assert lc.sum() == 0
        assert np.array_equal(thr.astype(np.int64), want), (q, s)


def test_sampling_stride_rejects_unfilterable(gpu):
    ref = synth.make_reference(200_000, 5, 0.0, 0.0)
    reads = synth.make_reads(ref, 10, 7, lengths=(100,))
    R = gpu.pack_reference(ref)
    # 100 bp, k = 5, q = 16: stride 3 leaves 29 sampled q-grams, 5 edits can touch 30
    with pytest.raises(gpu.PeanutError, match="stride"):
        gpu.index_reads(R, reads.seq, reads.offsets, 16, k=5, stride=3)


def test_result_heavy_submission_stays_within_budget(gpu):
    """Reads from a 300-copy family hit ~300 places each: the result rows held from the launches to
    the submission's assembly are reserved with the launches, so the engine's reserved device
    memory never exceeds its budget; the hits equal the oracle's."""
    ref = synth.make_reference(1_500_000, 97)
    fam = ref[-1000:-700].copy()
    rng = np.random.default_rng(3)
    for c in range(300):
        st = 4000 * c + int(rng.integers(0, 3000))
        ref[st:st + 300] = fam
    R = gpu.pack_reference(ref)
    reads = synth.make_reads(ref[:1_200_000], 3000, 98, lengths=(100,), rate_range=(0.0, 0.02))
    budget = 2 << 30
    res, st = run_engine(gpu, R, [reads, reads.slice(0, 1000)], ["all", "best"], executors=2, autotune=False,
                         max_reads=1500, hbm_budget=budget)
    assert st["hbm_reserved_peak"] <= budget, st["hbm_reserved_peak"]
    assert st["results"] > 20_000
    want = oracle.map_filter(ref, reads.seq, reads.offsets, [k_of(100)] * reads.n, 16, "all")
    assert np.array_equal(res[0], want)
