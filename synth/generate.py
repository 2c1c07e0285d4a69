"""Seeded synthetic references and reads (input generation only).

A thin ctypes wrapper over `synthgen.c`.  Every random number comes from one counter-based
generator, splitmix64 (Steele, Lea & Flood, OOPSLA 2014): draw i of stream s under seed S is
mix64(key(S, s) + (i + 1) * 0x9E3779B97F4A7C15), so the same inputs come out on any machine and
for any thread count.

Shapes follow the read-mapping workloads of Köster & Rahmann (PEANUT), Section "Results":
  * references: uniform i.i.d. ACGT, optionally with interspersed repeat families (consensus
    300 bp - 6 kbp log-uniform, 2-50 copies, 10-20 % per-copy substitution divergence) and
    low-complexity tandem runs (period 1-6, length 20-200);
  * reads: sampled at a uniform position on a uniform strand with substitutions and single-base
    insertions/deletions, or uniform random (unmappable) reads.
The datasets the paper measured on (GRCh37, exome runs, yeast) are not available; these
synthetic inputs stand in for them with the same read lengths, error rates and genome sizes.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synthgen.c")
_SO = os.path.join(_HERE, "_synthgen.so")
_lib = None

_COMP = np.zeros(256, dtype=np.uint8)
for _a, _b in zip(b"ACGTN", b"TGCAN"):
    _COMP[_a] = _b


def build(force: bool = False) -> str:
    """Compile synthgen.c into a shared object next to it (atomic replace)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
        os.close(fd)
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        c = ctypes
        lib.synth_key.restype = c.c_uint64
        lib.synth_key.argtypes = [c.c_uint64, c.c_uint64]
        lib.synth_draws.argtypes = [c.c_uint64, c.c_uint64, c.c_uint64, c.c_uint64, c.c_void_p]
        lib.synth_reference.argtypes = [c.c_void_p, c.c_uint64, c.c_uint64, c.c_double, c.c_double]
        lib.synth_read_lengths.argtypes = [c.c_uint64, c.c_uint64, c.c_void_p, c.c_int, c.c_void_p]
        lib.synth_reads.restype = c.c_int
        lib.synth_reads.argtypes = [c.c_void_p, c.c_uint64, c.c_uint64, c.c_uint64, c.c_void_p,
                                    c.c_void_p, c.c_int32, c.c_double, c.c_double, c.c_double,
                                    c.c_double, c.c_double, c.c_double, c.c_void_p, c.c_void_p,
                                    c.c_void_p, c.c_void_p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def counter_u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of splitmix64 stream `stream` under `seed`."""
    out = np.empty(count, dtype=np.uint64)
    _load().synth_draws(seed, stream, start, count, _ptr(out))
    return out


def revcomp_ascii(seq) -> np.ndarray:
    """Reverse complement of an ASCII ACGT sequence (bytes or uint8 array)."""
    a = np.frombuffer(seq, dtype=np.uint8) if isinstance(seq, (bytes, bytearray)) else np.asarray(seq)
    return _COMP[a[::-1]]


def make_reference(n: int, seed: int = 1403, repeat_frac: float = 0.0, tandem_frac: float = 0.0,
                   ) -> np.ndarray:
    """Reference of n bases (ASCII uint8): uniform background, repeat families, tandem runs."""
    out = np.empty(n, dtype=np.uint8)
    _load().synth_reference(_ptr(out), n, seed, repeat_frac, tandem_frac)
    return out


def uniform_reference(n: int, seed: int = 1403) -> np.ndarray:
    """n uniform i.i.d. ACGT bases (ASCII uint8)."""
    return make_reference(n, seed)


@dataclasses.dataclass
class Reads:
    """A read batch: concatenated ASCII bases and n+1 offsets, plus the planted truth.

    truth_end is the forward-coordinate end (0-based, inclusive) of the planted alignment, or -1
    for a uniform random read; truth_edits bounds the planted alignment's edit count from above;
    truth_strand is 0 for a read taken from the forward strand and 1 for the reverse strand.
    """
    seq: np.ndarray           # uint8 ASCII, concatenated
    offsets: np.ndarray       # uint64, n+1
    truth_end: np.ndarray     # int64
    truth_strand: np.ndarray  # uint8
    truth_edits: np.ndarray   # int32

    @property
    def n(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)

    def read(self, i: int) -> bytes:
        return self.seq[int(self.offsets[i]):int(self.offsets[i + 1])].tobytes()

    def subset(self, idx) -> "Reads":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths[idx]
        offs = np.zeros(idx.size + 1, dtype=np.uint64)
        offs[1:] = np.cumsum(lens)
        parts = [self.seq[int(self.offsets[i]):int(self.offsets[i + 1])] for i in idx]
        seq = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
        return Reads(seq, offs, self.truth_end[idx], self.truth_strand[idx], self.truth_edits[idx])

    def slice(self, a: int, b: int) -> "Reads":
        """Reads a..b-1 as a new batch (views where possible)."""
        o0, o1 = int(self.offsets[a]), int(self.offsets[b])
        return Reads(self.seq[o0:o1], (self.offsets[a:b + 1] - np.uint64(o0)).astype(np.uint64),
                     self.truth_end[a:b], self.truth_strand[a:b], self.truth_edits[a:b])


def make_reads(ref: np.ndarray, n_reads: int, seed: int, lengths=(100,), sub_rate=None,
               indel_rate=None, rate_range=None, sub_share=0.9, random_frac=0.0) -> Reads:
    """Sample `n_reads` reads from `ref` (ASCII uint8).

    Error model per source base: substitution `sub_rate`, indel `indel_rate` (insertion or
    deletion with equal odds); or, with `rate_range=(lo, hi)`, a per-read total rate
    e ~ U[lo, hi] split into substitutions (`sub_share`) and indels.  Lengths are drawn uniformly
    from `lengths`.  A fraction `random_frac` are uniform random (unmappable) reads.
    """
    lib = _load()
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    lengths = np.asarray(lengths, dtype=np.int32)
    lens = np.empty(n_reads, dtype=np.int32)
    lib.synth_read_lengths(n_reads, seed, _ptr(lengths), lengths.size, _ptr(lens))
    offsets = np.zeros(n_reads + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    seq = np.empty(int(offsets[-1]), dtype=np.uint8)
    te = np.empty(n_reads, dtype=np.int64)
    ts = np.empty(n_reads, dtype=np.uint8)
    tk = np.empty(n_reads, dtype=np.int32)
    lo, hi = rate_range if rate_range is not None else (0.0, 0.0)
    rc = lib.synth_reads(_ptr(ref), ref.size, n_reads, seed, _ptr(lens), _ptr(offsets),
                         int(lengths.max()), float(sub_rate or 0.0), float(indel_rate or 0.0),
                         float(lo), float(hi), float(sub_share), float(random_frac), _ptr(seq),
                         _ptr(te), _ptr(ts), _ptr(tk))
    if rc != 0:
        raise RuntimeError("read source window exhausted (reference too short?)")
    return Reads(seq, offsets, te, ts, tk)


def k_of_length(length, k):
    """Per-read error budget: a fixed int, or "5pct" = ceil(0.05 * length) in integers."""
    length = np.asarray(length, dtype=np.int64)
    if k == "5pct":
        return (5 * length + 99) // 100
    return np.full(length.shape, int(k), dtype=np.int64)


# The workloads.  Sizes, error models and parameters of each mapping run.
WORKLOADS = {
    "uniform_1mbp_10k": dict(ref_len=1_000_000, repeat_frac=0.0, tandem_frac=0.0, n_reads=10_000,
                             lengths=(100,), sub_rate=0.01, indel_rate=0.001, random_frac=0.0,
                             q=11, k=5, modes=("all",)),
    "repeat_100mbp_1m": dict(ref_len=100_000_000, repeat_frac=0.05, tandem_frac=0.01,
                             n_reads=1_000_000, lengths=(100,), rate_range=(0.01, 0.04),
                             random_frac=0.0, q=16, k=5, modes=("all", "best")),
    "human_3g1_10m": dict(ref_len=3_100_000_000, repeat_frac=0.45, tandem_frac=0.01,
                          n_reads=10_000_000, lengths=(100,), rate_range=(0.01, 0.04),
                          random_frac=0.05, q=16, k=5, modes=("all",), batch=1 << 20),
    "uneven_3g1_10m": dict(ref_len=3_100_000_000, repeat_frac=0.45, tandem_frac=0.01,
                           n_reads=10_000_000, lengths=(50, 75, 100, 150, 250),
                           rate_range=(0.02, 0.02), random_frac=0.0, q=12, k="5pct",
                           modes=("all",)),
    # request stream: Poisson arrivals (mean rate), request sizes log-uniform in [min, max] reads,
    # read lengths uniform in 75..250 bp, half the requests in best-stratum mode
    "serve_3g1": dict(ref_len=3_100_000_000, repeat_frac=0.45, tandem_frac=0.01,
                      lengths=tuple(range(75, 251)), rate_range=(0.01, 0.04), random_frac=0.0,
                      k="5pct", rate_per_s=50.0, req_min=1_000, req_max=1_000_000, n_requests=100,
                      modes=("all", "best")),
}


def uneven_batches(n_reads: int, seed: int, lo: int = 1 << 16, hi: int = 1 << 21):
    """Split n_reads into consecutive batches whose sizes are log-uniform in [lo, hi] (the last
    one takes the remainder); returns the batch boundaries."""
    rng = np.random.default_rng(seed)
    b = [0]
    while b[-1] < n_reads:
        size = int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))
        b.append(min(n_reads, b[-1] + size))
    return b


def request_stream(seed: int, n_requests: int, rate_per_s: float, req_min: int, req_max: int):
    """Arrival times (s, Poisson process), sizes (reads, log-uniform) and modes of a request
    stream."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_per_s, n_requests))
    sizes = np.exp(rng.uniform(np.log(req_min), np.log(req_max), n_requests)).round().astype(np.int64)
    modes = np.where(rng.random(n_requests) < 0.5, "all", "best")
    return arrivals, sizes, modes


def make_workload(name: str, ref_len: int | None = None, n_reads: int | None = None,
                  ref_seed: int = 1403, read_seed: int | None = None):
    """Reference, reads and parameters of a named workload, optionally scaled down."""
    w = dict(WORKLOADS[name])
    n = int(ref_len or w["ref_len"])
    nr = int(n_reads or w["n_reads"])
    ref = make_reference(n, ref_seed, w["repeat_frac"], w["tandem_frac"])
    seed = read_seed if read_seed is not None else 1706 + list(WORKLOADS).index(name)
    reads = make_reads(ref, nr, seed, lengths=w["lengths"], sub_rate=w.get("sub_rate"),
                       indel_rate=w.get("indel_rate"), rate_range=w.get("rate_range"),
                       random_frac=w["random_frac"])
    return ref, reads, w
