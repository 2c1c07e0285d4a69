"""PEANUT read-mapping oracle: TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline / reference arm may import
this package.  The CUDA library and its Python binding never import it; they share no code.

A ctypes wrapper over `peanut_oracle.c` (plain, slow, single-threaded C; see its header for the
definitions, each tied to its section of Köster & Rahmann, "Massively parallel read mapping on GPUs
with PEANUT") plus the closed-form index sizes of Section "The q-group index", paragraph "Size".

Hit sets are returned as a numpy structured array with fields read (u4), strand (u1: 0 = read,
1 = reverse complement of the read on the forward reference), end (i8: 0-based inclusive end in
forward coordinates) and dist (i4: edit distance), sorted by (read, strand, end).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "peanut_oracle.c")
_SO = os.path.join(_HERE, "_peanut_oracle.so")
_lib = None

HIT_DTYPE = np.dtype([("read", "<u4"), ("strand", "u1"), ("end", "<i8"), ("dist", "<i4")])
MODES = {"all": 0, "best": 1, "ends": 2}


def build(force: bool = False) -> str:
    """Compile the oracle into a shared object next to its source (atomic replace)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
        os.close(fd)
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        c = ctypes
        vp = c.c_void_p
        lib.oracle_semiglobal_column.restype = c.c_int
        lib.oracle_semiglobal_column.argtypes = [vp, c.c_int64, vp, c.c_int64, vp]
        lib.oracle_map_bruteforce.restype = vp
        lib.oracle_map_bruteforce.argtypes = [vp, c.c_int64, vp, vp, c.c_int64, vp, c.c_int, vp, c.c_int64]
        lib.oracle_map_filter.restype = vp
        lib.oracle_map_filter.argtypes = [vp, c.c_int64, vp, vp, c.c_int64, vp, c.c_int, c.c_int, vp, c.c_int64]
        lib.oracle_splitmix64.restype = c.c_uint64
        lib.oracle_splitmix64.argtypes = [c.c_uint64, c.c_uint64]
        lib.oracle_fnv1a64.restype = c.c_uint64
        lib.oracle_fnv1a64.argtypes = [vp, c.c_int64]
        lib.oracle_prepare_reference.restype = c.c_int64
        lib.oracle_prepare_reference.argtypes = [vp, c.c_int64, vp, c.c_int64, c.c_int64, c.c_uint64, vp, vp,
                                                 c.c_int64]
        lib.oracle_pair_hits.restype = c.c_int64
        lib.oracle_pair_hits.argtypes = [vp, vp, vp, vp, vp, c.c_int64, vp, c.c_int64, vp, c.c_int64, c.c_int64,
                                         c.c_int64, c.c_int64, c.c_int, vp, vp, vp, vp, vp, c.c_int64]
        lib.oracle_cigar.restype = c.c_int64
        lib.oracle_cigar.argtypes = [vp, c.c_int64, vp, c.c_int64, c.c_int32, vp, vp, c.c_int64]
        lib.oracle_prepare_reads.restype = c.c_int
        lib.oracle_prepare_reads.argtypes = [vp, vp, c.c_int64, c.c_uint64, vp]
        lib.oracle_hits_count.restype = c.c_int64
        lib.oracle_hits_count.argtypes = [vp]
        lib.oracle_hits_copy.argtypes = [vp, vp, vp, vp, vp]
        lib.oracle_hits_free.argtypes = [vp]
        lib.oracle_qgroup_build.restype = c.c_int64
        lib.oracle_qgroup_build.argtypes = [vp, vp, c.c_int64, c.c_int, c.c_int, vp, vp, vp, vp]
        lib.oracle_indexpair.argtypes = [vp, vp, vp, c.c_int, c.c_uint64, vp, vp]
        lib.oracle_canonical_text.restype = c.c_int64
        lib.oracle_canonical_text.argtypes = [vp, vp, c.c_int64, c.c_int, vp, vp]
        lib.oracle_frequent_qgrams.restype = c.c_int64
        lib.oracle_frequent_qgrams.argtypes = [vp, c.c_int64, c.c_int, c.c_int64, vp, vp, c.c_int64]
        lib.oracle_annotate.restype = c.c_int
        lib.oracle_annotate.argtypes = [vp, c.c_int64, vp, vp, c.c_int64, vp, vp, vp, vp, c.c_int64, vp, vp, vp,
                                        vp, c.c_int64]
        _lib = lib
    return _lib


def _bytes(x) -> np.ndarray:
    """The sequence as a contiguous uint8 array (a view of numpy input; no 3 GB copies)."""
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8)
    return np.ascontiguousarray(x, dtype=np.uint8)


_EMPTY = np.zeros(8, np.uint8)


def _p(a: np.ndarray) -> int:
    """Address of a contiguous array, for the ctypes calls (the caller keeps `a` alive)."""
    return a.ctypes.data if a.size else _EMPTY.ctypes.data


def _reads_args(seq, offsets):
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    return _bytes(seq), offs


def _collect(h) -> np.ndarray:
    lib = _load()
    if not h:
        raise ValueError("oracle rejected the input (non-ACGT base, bad q, or lemma threshold < 1)")
    try:
        n = lib.oracle_hits_count(h)
        r = np.empty(n, np.uint32)
        s = np.empty(n, np.uint8)
        e = np.empty(n, np.int64)
        d = np.empty(n, np.int32)
        if n:
            lib.oracle_hits_copy(h, r.ctypes.data, s.ctypes.data, e.ctypes.data, d.ctypes.data)
    finally:
        lib.oracle_hits_free(h)
    out = np.empty(n, HIT_DTYPE)
    out["read"], out["strand"], out["end"], out["dist"] = r, s, e, d
    return out


def semiglobal_column(pattern, ref) -> np.ndarray:
    """D[j] = E[m][j] of Section "Validation" for every end position j of `ref`."""
    P, R = _bytes(pattern), _bytes(ref)
    D = np.empty(max(len(R), 1), np.int32)
    if _load().oracle_semiglobal_column(_p(P), len(P), _p(R), len(R), D.ctypes.data) != 0:
        raise ValueError("non-ACGT character")
    return D[:len(R)]


def _kvec(k, n):
    k = np.asarray(k, dtype=np.int32)
    if k.ndim == 0:
        k = np.full(n, int(k), dtype=np.int32)
    return np.ascontiguousarray(k)


def _segs(segments):
    """Segments as a contiguous int64 (start, end) array and their count; None = the whole text."""
    if segments is None:
        return None, 0
    sg = np.ascontiguousarray(np.asarray(segments, dtype=np.int64).reshape(-1, 2))
    return sg, sg.shape[0]


def map_bruteforce(ref, seq, offsets, k, mode: str = "all", segments=None) -> np.ndarray:
    """Hit set by the definition: full semiglobal DP of every read and strand over `ref` (over each
    segment separately, the matrix restarting at its start, when `segments` is given)."""
    R = _bytes(ref)
    S, offs = _reads_args(seq, offsets)
    n = offs.size - 1
    kv = _kvec(k, n)
    sg, ns = _segs(segments)
    return _collect(_load().oracle_map_bruteforce(_p(R), len(R), _p(S), offs.ctypes.data, n, kv.ctypes.data,
                                                  MODES[mode], sg.ctypes.data if ns else None, ns))


def map_filter(ref, seq, offsets, k, q: int, mode: str = "all", segments=None) -> np.ndarray:
    """Hit set by the q-gram filter + windowed DP (equal to map_bruteforce when every t >= 1)."""
    R = _bytes(ref)
    S, offs = _reads_args(seq, offsets)
    n = offs.size - 1
    kv = _kvec(k, n)
    sg, ns = _segs(segments)
    return _collect(_load().oracle_map_filter(_p(R), len(R), _p(S), offs.ctypes.data, n, kv.ctypes.data,
                                              int(q), MODES[mode], sg.ctypes.data if ns else None, ns))


def splitmix64(seed: int, i: int) -> int:
    """Output number i (i >= 1) of SplitMix64 seeded with `seed`."""
    return int(_load().oracle_splitmix64(seed & (2 ** 64 - 1), i))


def fnv1a64(data) -> int:
    """FNV-1a 64 of a byte string."""
    b = _bytes(data)
    return int(_load().oracle_fnv1a64(_p(b), b.size))


def prepare_reference(seq, contig_starts=(0,), gap_min: int = 16, seed: int = 0):
    """(text, segments): the reference with every N replaced by its seeded base, and its
    segments as an (s, 2) int64 array of [start, end) (contigs cut at runs of >= gap_min Ns)."""
    R = _bytes(seq)
    cs = np.ascontiguousarray(np.asarray(contig_starts, dtype=np.int64))
    text = np.empty(max(R.size, 1), np.uint8)
    cap = 16
    while True:
        sg = np.empty((cap, 2), np.int64)
        ns = _load().oracle_prepare_reference(_p(R), R.size, _p(cs), cs.size, gap_min, seed & (2 ** 64 - 1),
                                              text.ctypes.data, sg.ctypes.data, cap)
        if ns == -2:
            cap *= 4
            continue
        if ns < 0:
            raise ValueError("bad reference byte or contig list")
        return text[:R.size], sg[:ns].copy()


def prepare_reads(seq, offsets, seed: int = 0) -> np.ndarray:
    """The reads upper-cased with every N replaced by its seeded base."""
    S, offs = _reads_args(seq, offsets)
    out = np.empty(max(S.size, 1), np.uint8)
    if _load().oracle_prepare_reads(_p(S), offs.ctypes.data, offs.size - 1, seed & (2 ** 64 - 1),
                                    out.ctypes.data) != 0:
        raise ValueError("bad read byte")
    return out[:S.size]


def annotate(ref, seq, offsets, hits: np.ndarray, segments=None):
    """Per hit (a hit set grouped by read): the leftmost alignment start (backward DP, Section
    "Validation"), the hit-rank and the mapping quality (Section "Postprocessing").  Returns
    (start int64, rank uint32, mapq int32)."""
    R = _bytes(ref)
    S, offs = _reads_args(seq, offsets)
    n = offs.size - 1
    hr = np.ascontiguousarray(hits["read"], np.uint32)
    hs = np.ascontiguousarray(hits["strand"], np.uint8)
    he = np.ascontiguousarray(hits["end"], np.int64)
    hd = np.ascontiguousarray(hits["dist"], np.int32)
    nh = hr.size
    start = np.empty(max(nh, 1), np.int64)
    rank = np.empty(max(nh, 1), np.uint32)
    mapq = np.empty(max(nh, 1), np.int32)
    sg, ns = _segs(segments)
    if _load().oracle_annotate(_p(R), len(R), _p(S), offs.ctypes.data, n, _p(hr), _p(hs), _p(he), _p(hd), nh,
                               start.ctypes.data, rank.ctypes.data, mapq.ctypes.data,
                               sg.ctypes.data if ns else None, ns) != 0:
        raise ValueError("bad input to annotate")
    return start[:nh], rank[:nh], mapq[:nh]


def qgroup_build(codes, payload, q: int, w: int = 32):
    """Algorithm 1 over a text of q-gram codes.  Returns (I, S, Sp, O, distinct) with Sp cut to
    distinct + 1 entries (the last one is the sentinel |T|)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    payload = np.ascontiguousarray(payload, dtype=np.uint64)
    T = codes.size
    ng = ((1 << (2 * q)) + w - 1) // w
    I = np.empty(ng, np.uint64)
    S = np.empty(ng, np.uint64)
    Sp = np.empty(T + 1, np.uint64)
    O = np.empty(max(T, 1), np.uint64)
    d = _load().oracle_qgroup_build(codes.ctypes.data, payload.ctypes.data, T, q, w, I.ctypes.data,
                                    S.ctypes.data, Sp.ctypes.data, O.ctypes.data)
    if d < 0:
        raise ValueError("bad q or w")
    return I, S, Sp[:d + 1].copy(), O[:T], int(d)


def indexpair(I, S, Sp, w: int, g: int):
    """INDEXPAIR(g) of Section "Filtration"; (0, 0) when g does not occur."""
    a = ctypes.c_uint64()
    b = ctypes.c_uint64()
    Sp_full = np.ascontiguousarray(np.append(Sp, 0), dtype=np.uint64)
    _load().oracle_indexpair(np.ascontiguousarray(I).ctypes.data, np.ascontiguousarray(S).ctypes.data,
                             Sp_full.ctypes.data, w, int(g), ctypes.byref(a), ctypes.byref(b))
    return int(a.value), int(b.value)


def canonical_text(seq, offsets, q: int):
    """(codes, payload) of every read q-gram: canonical code min(g, revcomp g) and the label
    (read << 9) | (g != canonical) << 8 | offset."""
    S, offs = _reads_args(seq, offsets)
    n = offs.size - 1
    lens = np.diff(offs)
    total = int(np.maximum(lens - q + 1, 0).sum())
    codes = np.empty(max(total, 1), np.uint64)
    payload = np.empty(max(total, 1), np.uint64)
    got = _load().oracle_canonical_text(_p(S), offs.ctypes.data, n, q, codes.ctypes.data, payload.ctypes.data)
    if got < 0:
        raise ValueError("bad input")
    return codes[:got], payload[:got]


def frequent_qgrams(ref, q: int, cap: int, max_out: int = 1 << 20):
    """Canonical q-grams occurring more than `cap` times in `ref`: (codes, counts) by code."""
    R = _bytes(ref)
    codes = np.empty(max_out, np.uint64)
    counts = np.empty(max_out, np.int64)
    n = _load().oracle_frequent_qgrams(_p(R), len(R), q, cap, codes.ctypes.data, counts.ctypes.data, max_out)
    if n < 0:
        raise ValueError("bad input")
    if n > max_out:
        return frequent_qgrams(ref, q, cap, max_out=int(n))
    return codes[:n].copy(), counts[:n].copy()


# ---- closed-form sizes, Section "The q-group index", paragraph "Size" (in words) ----

def qgroup_index_words(q: int, T: int, w: int = 32) -> float:
    """Upper bound on the q-group index size: 2/w * 4^q + min(4^q, |T|) + |T| words."""
    return 2.0 / w * 4 ** q + min(4 ** q, T) + T


def qgram_index_words(q: int, T: int) -> float:
    """Size of a plain q-gram index (address table + position table): 4^q + |T| words."""
    return float(4 ** q + T)


def lemma_threshold(m: int, q: int, k: int) -> int:
    """q-gram lemma: an alignment with at most k errors keeps at least m + 1 - q(k + 1) of the
    read's q-grams intact (Section "The q-group index", paragraph on the choice of q)."""
    return m + 1 - q * (k + 1)


def sort_hits(h: np.ndarray) -> np.ndarray:
    """Hits in (read, strand, end) order."""
    return h[np.lexsort((h["end"], h["strand"], h["read"]))]


PAIR_DTYPE = np.dtype([("i1", "<i8"), ("i2", "<i8"), ("score", "<i8"), ("rank", "<u4"), ("mapq", "<i4")])


def pair_hits(hits: np.ndarray, starts, offsets, n_ref: int, min_insert: int, max_insert: int,
              mode: str = "all", contig_starts=(0,)) -> np.ndarray:
    """Proper pairs of mates 2p / 2p + 1 (Section "Postprocessing", paired-end mode; readings in
    oracle_pair_hits): hit indices i1 (mate 1) and i2 (mate 2), summed-identity numerator score,
    rank and quality; mode "all" or "best"."""
    hr = np.ascontiguousarray(hits["read"], np.uint32)
    hs = np.ascontiguousarray(hits["strand"], np.uint8)
    he = np.ascontiguousarray(hits["end"], np.int64)
    hd = np.ascontiguousarray(hits["dist"], np.int32)
    st = np.ascontiguousarray(starts, np.int64)
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    cs = np.ascontiguousarray(np.asarray(contig_starts, dtype=np.int64))
    cap = max(16, hr.size)
    while True:
        o1, o2, sc = (np.empty(cap, np.int64) for _ in range(3))
        rk = np.empty(cap, np.uint32)
        mq = np.empty(cap, np.int32)
        got = _load().oracle_pair_hits(_p(hr), _p(hs), _p(he), _p(st), _p(hd), hr.size, offs.ctypes.data,
                                       offs.size - 1, cs.ctypes.data, cs.size, int(n_ref), int(min_insert),
                                       int(max_insert), {"all": 0, "best": 1}[mode], o1.ctypes.data, o2.ctypes.data,
                                       sc.ctypes.data, rk.ctypes.data, mq.ctypes.data, cap)
        if got < 0:
            raise ValueError("bad input to pair_hits")
        if got <= cap:
            out = np.empty(got, PAIR_DTYPE)
            out["i1"], out["i2"], out["score"], out["rank"], out["mapq"] = o1[:got], o2[:got], sc[:got], rk[:got], mq[:got]
            return out
        cap = int(got)


_COMP = bytes.maketrans(b"ACGT", b"TGCA")


def cigar(pattern, text, dist: int) -> str:
    """The hit's alignment (readings in oracle_cigar) as an extended CIGAR string: runs of
    '=' (match), 'X' (mismatch), 'I' (read base only), 'D' (reference base only)."""
    P, T = _bytes(pattern), _bytes(text)
    cap = P.size + T.size + 1
    ops = np.empty(cap, np.uint8)
    lens = np.empty(cap, np.int32)
    n = _load().oracle_cigar(_p(P), P.size, _p(T), T.size, int(dist), ops.ctypes.data, lens.ctypes.data, cap)
    if n < 0:
        raise ValueError("the distance is not the edit distance of pattern and text")
    return "".join(f"{int(l)}{chr(o)}" for o, l in zip(ops[:n], lens[:n]))


def alignments(ref, seq, offsets, hits: np.ndarray, starts) -> list:
    """The CIGAR string of every hit (pattern: the read, or its reverse complement for strand 1;
    text: ref[start..end])."""
    R = _bytes(ref)
    S, offs = _reads_args(seq, offsets)
    out = []
    for h, st in zip(hits, starts):
        r = int(h["read"])
        read = bytes(S[offs[r]:offs[r + 1]])
        pat = read[::-1].translate(_COMP) if h["strand"] else read
        out.append(cigar(pat, bytes(R[int(st):int(h["end"]) + 1]), int(h["dist"])))
    return out
