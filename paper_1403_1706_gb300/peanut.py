"""Python binding of libpeanut (include/peanut.h): argument marshalling only.

Every function here forwards to the C ABI of the same name; all mapping work runs in the CUDA
library.  There is no CPU fallback: if libpeanut.so is missing or no GPU is present, calls raise.

Hit sets come back as numpy structured arrays with fields read (u4), strand (u1), end (i8) and
dist (i4), sorted by (read, strand, end) -- the layout of peanut_hits widened for comparison.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_float, c_int, c_int32, c_size_t, c_uint8, c_uint16
from ctypes import c_uint32, c_uint64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpeanut.so")
HIT_DTYPE = np.dtype([("read", "<u4"), ("strand", "u1"), ("end", "<i8"), ("dist", "<i4")])
MODES = {"all": 0, "best": 1}
K_FROM_PERMILLE = 0xFFFFFFFF

_lib = None


class PeanutError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"peanut status {status}: {msg}")
        self.status = status


class Params(Structure):
    _fields_ = [("q", c_uint32), ("k_fixed", c_uint32), ("k_permille", c_uint32), ("freq_cap", c_uint32),
                ("stride", c_uint32), ("stream", c_void_p), ("ref_index", c_uint32), ("index_layout", c_uint32)]


class Hits(Structure):
    _fields_ = [("n", c_uint64), ("read_id", POINTER(c_uint32)), ("strand", POINTER(c_uint8)),
                ("end_pos", POINTER(c_uint64)), ("dist", POINTER(c_uint8))]


class DeviceHitsStruct(Structure):
    _fields_ = [("n", c_uint64), ("read_id", c_void_p), ("strand", c_void_p), ("end_pos", c_void_p),
                ("dist", c_void_p)]


class DevicePairsStruct(Structure):
    _fields_ = [("n", c_uint64), ("i1", c_void_p), ("i2", c_void_p), ("score", c_void_p), ("rank", c_void_p),
                ("mapq", c_void_p)]


class MapStats(Structure):
    _fields_ = [("hits", c_uint64), ("candidates", c_uint64), ("candidate_columns", c_uint64),
                ("results", c_uint64), ("lowcx_reads", c_uint64), ("lowcx_ranges", c_uint64),
                ("scan_retries", c_uint64),
                ("present_probes", c_uint64), ("candidate_word_columns", c_uint64),
                ("ms_scan", c_float), ("ms_bin", c_float), ("ms_windows", c_float), ("ms_verify", c_float),
                ("ms_output", c_float), ("ms_scan_kernel", c_float), ("ms_verify_kernel", c_float),
                ("ms_windows_sweep", c_float), ("ms_lowcx", c_float), ("ms_compact", c_float),
                ("ms_probe_kernel", c_float), ("ms_windows_med", c_float), ("ms_windows_big", c_float),
                ("med_reads", c_uint64), ("big_reads", c_uint64), ("lowcx_rest_segments", c_uint64),
                ("lowcx_serial_segments", c_uint64), ("useful_columns", c_uint64),
                ("prefilter_columns", c_uint64), ("filter_positions", c_uint64), ("filter_live", c_uint64),
                ("ms_filter_kernel", c_float), ("graph_segments", c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class EngineParams(Structure):
    _fields_ = [("k_fixed", c_uint32), ("k_permille", c_uint32), ("executors", c_uint32), ("max_reads", c_uint32),
                ("autotune", c_uint32), ("fixed_q", c_uint32), ("hbm_budget", c_uint64), ("graphs", c_uint32)]


class EngineClass(Structure):
    _fields_ = [("q_class", c_uint32), ("q", c_uint32), ("stride", c_uint32), ("freq_cap", c_uint32),
                ("launches", c_uint64), ("reads", c_uint64), ("bytes_per_read", c_uint64),
                ("tuned_ms_per_mread", c_float), ("tune_candidates", c_uint32)]


class EngineStats(Structure):
    _fields_ = [("submissions", c_uint64), ("completed", c_uint64), ("reads", c_uint64), ("launches", c_uint64),
                ("tuning_launches", c_uint64), ("hbm_budget", c_uint64), ("hbm_reserved_peak", c_uint64),
                ("n_classes", c_uint32), ("cls", EngineClass * 16),
                ("map_runs", c_uint64), ("hits", c_uint64), ("candidates", c_uint64),
                ("candidate_word_columns", c_uint64), ("present_probes", c_uint64), ("results", c_uint64),
                ("bases_scanned", c_uint64), ("ms_verify_kernel", ctypes.c_double),
                ("ms_scan_kernel", ctypes.c_double), ("ms_probe_kernel", ctypes.c_double),
                ("ms_admit", ctypes.c_double), ("ms_launch", ctypes.c_double), ("ms_assemble", ctypes.c_double),
                ("ms_download", ctypes.c_double), ("pageable_result_blocks", c_uint64),
                ("candidate_columns", c_uint64), ("useful_columns", c_uint64),
                ("filter_positions", c_uint64), ("ms_filter_kernel", ctypes.c_double),
                ("graph_segments", c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, c_void_p)


def load():
    """Loads libpeanut.so (built by paper_1403_1706_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run paper_1403_1706_gb300.build.build() first "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    st = c_int
    sig = {
        "peanut_last_error": (c_char_p, []),
        "peanut_kernel_launches": (c_uint64, []),
        "peanut_set_allocator": (st, [ALLOC_FN, RELEASE_FN, c_void_p]),
        "peanut_pack_reference": (st, [c_void_p, c_uint64, c_void_p, POINTER(c_void_p)]),
        "peanut_pack_reference_contigs": (st, [c_void_p, c_uint64, c_void_p, c_uint32, c_uint32, c_uint64, c_void_p,
                                               POINTER(c_void_p)]),
        "peanut_ref_segments": (st, [c_void_p, POINTER(c_uint64), c_void_p, c_void_p]),
        "peanut_ref_length": (c_uint64, [c_void_p]),
        "peanut_index_reads": (st, [c_void_p, c_void_p, c_void_p, c_uint32, POINTER(Params), POINTER(c_void_p)]),
        "peanut_index_reads_device": (st, [c_void_p, c_void_p, c_void_p, c_uint32, c_uint64, POINTER(Params),
                                           POINTER(c_void_p)]),
        "peanut_map": (st, [c_void_p, c_void_p, c_int, POINTER(POINTER(Hits))]),
        "peanut_map_device": (st, [c_void_p, c_void_p, c_int, POINTER(POINTER(DeviceHitsStruct))]),
        "peanut_download_hits": (st, [POINTER(DeviceHitsStruct), c_void_p, POINTER(POINTER(Hits))]),
        "peanut_get_map_stats": (st, [c_void_p, POINTER(MapStats)]),
        "peanut_free": (None, [c_void_p]),
        "peanut_index_sizes": (st, [c_void_p, POINTER(c_uint64), POINTER(c_uint64), POINTER(c_uint64)]),
        "peanut_export_index": (st, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "peanut_export_read_params": (st, [c_void_p, c_void_p, c_void_p]),
        "peanut_export_candidates": (st, [c_void_p, POINTER(c_uint64), c_void_p, c_void_p, c_void_p, c_void_p]),
        "peanut_debug_bitvector_columns": (st, [c_void_p, c_void_p, c_uint32, c_void_p, c_void_p, c_void_p,
                                                c_void_p]),
        "peanut_bitvector_columns_noalloc": (st, [c_void_p, c_void_p, c_uint32, c_void_p, c_void_p, c_void_p,
                                                  c_void_p]),
        "peanut_annotate_hits": (st, [c_void_p, c_void_p, POINTER(DeviceHitsStruct), c_void_p, c_void_p, c_void_p]),
        "peanut_index_reference": (st, [c_void_p, c_uint32, c_void_p]),
        "peanut_batch_max_k": (c_uint32, [c_void_p]),
        "peanut_hit_alignments": (st, [c_void_p, c_void_p, POINTER(DeviceHitsStruct), c_void_p, c_uint32, c_void_p,
                                       c_void_p]),
        "peanut_pair_hits": (st, [c_void_p, c_void_p, POINTER(DeviceHitsStruct), c_void_p, c_uint32, c_uint32, c_int,
                                  POINTER(POINTER(DevicePairsStruct))]),
        "peanut_download_pairs": (st, [POINTER(DevicePairsStruct), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_void_p]),
        "peanut_int_peak": (st, [c_uint32, c_uint32, c_void_p, POINTER(ctypes.c_double), POINTER(c_uint64),
                                 POINTER(c_uint32), POINTER(c_uint32)]),
        "peanut_engine_create": (st, [c_void_p, POINTER(EngineParams), POINTER(c_void_p)]),
        "peanut_engine_submit": (st, [c_void_p, c_void_p, c_void_p, c_uint32, c_int, POINTER(c_uint64)]),
        "peanut_engine_submit_device": (st, [c_void_p, c_void_p, c_void_p, c_uint32, c_uint64, c_int,
                                             POINTER(c_uint64)]),
        "peanut_engine_wait": (st, [c_void_p, c_uint64, ctypes.c_int64, POINTER(POINTER(Hits))]),
        "peanut_engine_wait_device": (st, [c_void_p, c_uint64, ctypes.c_int64,
                                           POINTER(POINTER(DeviceHitsStruct))]),
        "peanut_engine_get_stats": (st, [c_void_p, POINTER(EngineStats)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    # device memory of the calls made from Python comes from PyTorch's caching allocator (the
    # engines' own threads keep CUDA's stream-ordered pool); PEANUT_DEVICE_ALLOCATOR=cuda opts out
    if os.environ.get("PEANUT_DEVICE_ALLOCATOR", "torch") != "cuda":
        try:
            import torch
            if torch.cuda.is_available():
                use_torch_allocator()
        except ImportError:
            pass
    return lib


def _check(status: int):
    if status != 0:
        raise PeanutError(status, load().peanut_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _host_u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(x, dtype=np.uint8)
    return np.ascontiguousarray(x, dtype=np.uint8)


# ---- allocator -----------------------------------------------------------------------------

_alloc_keep = []  # every callback pair ever installed: objects made under it may still be freed


def use_torch_allocator():
    """Routes the library's device allocations through PyTorch's caching allocator."""
    import torch

    def _alloc(size, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(), stream or 0))
        except Exception:
            return None

    def _release(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, r = ALLOC_FN(_alloc), RELEASE_FN(_release)
    _alloc_keep.append((a, r))
    _check(load().peanut_set_allocator(a, r, None))


def use_default_allocator():
    _check(load().peanut_set_allocator(ALLOC_FN(), RELEASE_FN(), None))


# ---- objects -------------------------------------------------------------------------------

class _Handle:
    def __init__(self, ptr):
        self.ptr = ptr

    def free(self):
        if self.ptr:
            load().peanut_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Reference(_Handle):
    @property
    def length(self) -> int:
        return int(load().peanut_ref_length(self.ptr))


class ReadBatch(_Handle):
    def __init__(self, ptr, ref: Reference, n_reads: int):
        super().__init__(ptr)
        self.ref = ref  # keeps the reference alive while the batch exists
        self.n_reads = n_reads


DEFAULT_GAP_MIN = 16


def pack_reference(seq, stream=None, contigs=None, gap_min: int = DEFAULT_GAP_MIN, seed: int = 0) -> Reference:
    """peanut_pack_reference (one contig) or, with `contigs` (ascending start positions, the first
    0), peanut_pack_reference_contigs: ASCII reference (bytes or uint8 array; A/C/G/T/N in either
    case) -> resident packed reference.  N takes a seeded base; runs of >= gap_min Ns and contig
    boundaries cut the reference into segments no hit leaves."""
    a = _host_u8(seq)
    out = c_void_p()
    if contigs is None and gap_min == DEFAULT_GAP_MIN and seed == 0:
        _check(load().peanut_pack_reference(a.ctypes.data, a.size, _stream_ptr(stream), ctypes.byref(out)))
    else:
        cs = np.ascontiguousarray(np.asarray([0] if contigs is None else contigs, dtype=np.uint64))
        _check(load().peanut_pack_reference_contigs(a.ctypes.data, a.size, cs.ctypes.data, cs.size, int(gap_min),
                                                    int(seed) & (2 ** 64 - 1), _stream_ptr(stream),
                                                    ctypes.byref(out)))
    return Reference(out.value)


def ref_segments(ref: Reference) -> np.ndarray:
    """peanut_ref_segments: the reference's segments as an (s, 2) uint64 array of [start, end)."""
    n = c_uint64()
    _check(load().peanut_ref_segments(ref.ptr, ctypes.byref(n), None, None))
    st = np.empty(n.value, np.uint64)
    en = np.empty(n.value, np.uint64)
    if n.value:
        _check(load().peanut_ref_segments(ref.ptr, ctypes.byref(n), st.ctypes.data, en.ctypes.data))
    return np.stack([st, en], axis=1)


INDEX_LAYOUTS = {"interleaved": 0, "sampled_s": 1, "w64": 2}


def make_params(q: int, k=None, k_permille=None, freq_cap: int = 0, stream=None, stride: int = 1,
                ref_index: bool = False, layout: str = "interleaved") -> Params:
    if k is None and k_permille is None:
        raise ValueError("give k or k_permille")
    return Params(q, K_FROM_PERMILLE if k is None else int(k), int(k_permille or 0), int(freq_cap),
                  int(stride), _stream_ptr(stream), 1 if ref_index else 0, INDEX_LAYOUTS[layout])


def index_reference(ref: "Reference", q: int, stream=None) -> None:
    """peanut_index_reference: build (once) the reference's own q-group index at this q."""
    _check(load().peanut_index_reference(ref.ptr, int(q), _stream_ptr(stream)))


def index_reads(ref: Reference, seq, offsets, q: int, k=None, k_permille=None, freq_cap: int = 0,
                stream=None, stride: int = 1, ref_index: bool = False, layout: str = "interleaved") -> ReadBatch:
    """peanut_index_reads: host reads (concatenated ASCII + n+1 offsets) -> indexed batch."""
    s = _host_u8(seq)
    o = np.ascontiguousarray(offsets, dtype=np.uint64)
    p = make_params(q, k, k_permille, freq_cap, stream, stride, ref_index, layout)
    out = c_void_p()
    _check(load().peanut_index_reads(ref.ptr, s.ctypes.data, o.ctypes.data, o.size - 1, ctypes.byref(p),
                                     ctypes.byref(out)))
    return ReadBatch(out.value, ref, o.size - 1)


def index_reads_device(ref: Reference, d_seq, d_offsets, q: int, k=None, k_permille=None, freq_cap: int = 0,
                       stream=None, stride: int = 1, ref_index: bool = False,
                       layout: str = "interleaved") -> ReadBatch:
    """peanut_index_reads_device: reads already in device memory (torch uint8 / int64 tensors)."""
    p = make_params(q, k, k_permille, freq_cap, stream, stride, ref_index, layout)
    out = c_void_p()
    n = int(d_offsets.numel()) - 1
    _check(load().peanut_index_reads_device(ref.ptr, d_seq.data_ptr(), d_offsets.data_ptr(), n,
                                            int(d_seq.numel()), ctypes.byref(p), ctypes.byref(out)))
    return ReadBatch(out.value, ref, n)


def _hits_to_numpy(hp) -> np.ndarray:
    h = hp.contents
    n = int(h.n)
    out = np.empty(n, HIT_DTYPE)
    if n:
        out["read"] = np.ctypeslib.as_array(h.read_id, (n,))
        out["strand"] = np.ctypeslib.as_array(h.strand, (n,))
        out["end"] = np.ctypeslib.as_array(h.end_pos, (n,)).astype(np.int64)
        out["dist"] = np.ctypeslib.as_array(h.dist, (n,))
    return out


class HostHits:
    """A peanut_hits result held by the library: numpy views of its four arrays (read, strand,
    end, dist), valid while this object lives."""

    def __init__(self, hp):
        self._hp = hp
        h = hp.contents
        self.n = int(h.n)
        n = self.n
        self.read = np.ctypeslib.as_array(h.read_id, (n,)) if n else np.empty(0, np.uint32)
        self.strand = np.ctypeslib.as_array(h.strand, (n,)) if n else np.empty(0, np.uint8)
        self.end = np.ctypeslib.as_array(h.end_pos, (n,)) if n else np.empty(0, np.uint64)
        self.dist = np.ctypeslib.as_array(h.dist, (n,)) if n else np.empty(0, np.uint8)

    def free(self):
        if self._hp is not None:
            load().peanut_free(ctypes.cast(self._hp, c_void_p))
            self._hp = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def map_arrays(ref: Reference, batch: ReadBatch, mode: str = "all") -> HostHits:
    """peanut_map without a copy: the library's host arrays as numpy views."""
    hp = POINTER(Hits)()
    _check(load().peanut_map(ref.ptr, batch.ptr, MODES[mode], ctypes.byref(hp)))
    return HostHits(hp)


def map(ref: Reference, batch: ReadBatch, mode: str = "all") -> np.ndarray:
    """peanut_map: the batch's hit set on the host."""
    hp = POINTER(Hits)()
    _check(load().peanut_map(ref.ptr, batch.ptr, MODES[mode], ctypes.byref(hp)))
    try:
        return _hits_to_numpy(hp)
    finally:
        load().peanut_free(ctypes.cast(hp, c_void_p))


class DeviceHits(_Handle):
    """peanut_device_hits: result arrays left in device memory."""

    def __init__(self, hp):
        super().__init__(ctypes.cast(hp, c_void_p).value)
        self._hp = hp

    @property
    def n(self) -> int:
        return int(self._hp.contents.n)

    def to_numpy(self, stream=None) -> np.ndarray:
        out = POINTER(Hits)()
        _check(load().peanut_download_hits(self._hp, _stream_ptr(stream), ctypes.byref(out)))
        try:
            return _hits_to_numpy(out)
        finally:
            load().peanut_free(ctypes.cast(out, c_void_p))


def map_device(ref: Reference, batch: ReadBatch, mode: str = "all") -> DeviceHits:
    hp = POINTER(DeviceHitsStruct)()
    _check(load().peanut_map_device(ref.ptr, batch.ptr, MODES[mode], ctypes.byref(hp)))
    return DeviceHits(hp)


def annotate_hits(ref: Reference, batch: ReadBatch, hits: DeviceHits):
    """peanut_annotate_hits on a device hit list of the batch: (start, rank, mapq) as torch device
    tensors (int64, int32 holding the uint32 ranks, uint8), one entry per hit."""
    import torch
    n = hits.n
    dev = torch.device("cuda", torch.cuda.current_device())
    start = torch.empty(max(n, 1), dtype=torch.int64, device=dev)
    rank = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    mapq = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
    _check(load().peanut_annotate_hits(ref.ptr, batch.ptr, hits._hp, start.data_ptr(), rank.data_ptr(),
                                       mapq.data_ptr()))
    return start[:n], rank[:n], mapq[:n]


CIGAR_OPS = "=XID"


def hit_alignments(ref: Reference, batch: ReadBatch, hits: DeviceHits, start, ops_per_hit: int = 0):
    """peanut_hit_alignments: the alignment of every hit as (ops, nops) torch device tensors
    (int32 words len << 2 | code, ops_per_hit per hit; uint16 run counts stored in int16).
    ops_per_hit 0 = 2 k + 1 for the batch's largest k."""
    import torch
    n = hits.n
    cap = int(ops_per_hit) or 2 * int(load().peanut_batch_max_k(batch.ptr)) + 1
    dev = torch.device("cuda", torch.cuda.current_device())
    ops = torch.empty(max(n, 1) * cap, dtype=torch.int32, device=dev)
    nops = torch.empty(max(n, 1), dtype=torch.int16, device=dev)
    _check(load().peanut_hit_alignments(ref.ptr, batch.ptr, hits._hp, start.data_ptr() if n else None, cap,
                                        ops.data_ptr(), nops.data_ptr()))
    return ops[:n * cap].view(n, cap), nops[:n]


def cigars(ops, nops) -> list:
    """The extended CIGAR strings of hit_alignments' output (host conversion of device arrays)."""
    o = ops.cpu().numpy().view(np.uint32)
    c = nops.cpu().numpy().view(np.uint16)
    return ["".join(f"{w >> 2}{CIGAR_OPS[w & 3]}" for w in o[x, :c[x]]) for x in range(c.size)]


PAIR_DTYPE = np.dtype([("i1", "<u8"), ("i2", "<u8"), ("score", "<u4"), ("rank", "<u4"), ("mapq", "u1")])


def pair_hits(ref: Reference, batch: ReadBatch, hits: DeviceHits, start, min_insert: int, max_insert: int,
              mode: str = "all", stream=None) -> np.ndarray:
    """peanut_pair_hits + peanut_download_pairs: the proper pairs of mates 2p / 2p + 1 of a
    paired batch, given its device hit list and their starts (a torch int64 device tensor from
    annotate_hits), as a host structured array (i1, i2, score, rank, mapq)."""
    hp = POINTER(DevicePairsStruct)()
    _check(load().peanut_pair_hits(ref.ptr, batch.ptr, hits._hp, start.data_ptr() if hits.n else None,
                                   int(min_insert), int(max_insert), MODES[mode], ctypes.byref(hp)))
    try:
        n = int(hp.contents.n)
        out = np.empty(n, PAIR_DTYPE)
        cols = [np.empty(n, out.dtype[f]) for f in out.dtype.names]
        if n:
            _check(load().peanut_download_pairs(hp, _stream_ptr(stream), *[c.ctypes.data for c in cols]))
        for f, c in zip(out.dtype.names, cols):
            out[f] = c
        return out
    finally:
        load().peanut_free(ctypes.cast(hp, c_void_p))


def kernel_launches() -> int:
    """peanut_kernel_launches: kernels launched by the library so far in this process."""
    return int(load().peanut_kernel_launches())


INT_PEAK_KINDS = {"lop3": 0, "shf": 1, "iadd": 2, "imad": 3, "popc": 4, "myers_w1": 5, "myers_w2": 6,
                  "probe_l2": 7, "probe_hbm": 8}


def int_peak(kind: str, iters: int, stream=None) -> dict:
    """peanut_int_peak: one timed microbenchmark launch; ops per second of the given kind."""
    ms, ops, g, b = ctypes.c_double(), c_uint64(), c_uint32(), c_uint32()
    _check(load().peanut_int_peak(INT_PEAK_KINDS[kind], int(iters), _stream_ptr(stream), ctypes.byref(ms),
                                  ctypes.byref(ops), ctypes.byref(g), ctypes.byref(b)))
    return {"kind": kind, "ms": ms.value, "ops": ops.value, "ops_per_s": ops.value / (ms.value / 1e3),
            "grid": g.value, "block": b.value}


def get_map_stats(batch: ReadBatch) -> dict:
    s = MapStats()
    _check(load().peanut_get_map_stats(batch.ptr, ctypes.byref(s)))
    return s.as_dict()


# ---- introspection -------------------------------------------------------------------------

def index_sizes(batch: ReadBatch):
    a, b, c = c_uint64(), c_uint64(), c_uint64()
    _check(load().peanut_index_sizes(batch.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return int(a.value), int(b.value), int(c.value)


def export_index(batch: ReadBatch):
    """(I, S, Sp, O) of the batch's q-group index as numpy uint32 arrays."""
    ng, nd, ni = index_sizes(batch)
    I = np.empty(ng, np.uint32)
    S = np.empty(ng, np.uint32)
    Sp = np.empty(nd + 1, np.uint32)
    O = np.empty(max(ni, 1), np.uint32)
    _check(load().peanut_export_index(batch.ptr, I.ctypes.data, S.ctypes.data, Sp.ctypes.data, O.ctypes.data))
    return I, S, Sp, O[:ni]


def export_read_params(batch: ReadBatch):
    thr = np.empty(batch.n_reads, np.uint16)
    lc = np.empty(batch.n_reads, np.uint8)
    _check(load().peanut_export_read_params(batch.ptr, thr.ctypes.data, lc.ctypes.data))
    return thr, lc


def export_candidates(batch: ReadBatch):
    n = c_uint64(0)
    _check(load().peanut_export_candidates(batch.ptr, ctypes.byref(n), None, None, None, None))
    k = int(n.value)
    r = np.empty(max(k, 1), np.uint32)
    s = np.empty(max(k, 1), np.uint8)
    lo = np.empty(max(k, 1), np.uint64)
    hi = np.empty(max(k, 1), np.uint64)
    if k:
        _check(load().peanut_export_candidates(batch.ptr, ctypes.byref(n), r.ctypes.data, s.ctypes.data,
                                               lo.ctypes.data, hi.ctypes.data))
    return r[:k], s[:k], lo[:k].astype(np.int64), hi[:k].astype(np.int64)


def bitvector_columns(patterns, texts, stream=None):
    """peanut_debug_bitvector_columns: D columns of (pattern, text) pairs, one int32 array each."""
    pats = [bytes(p) for p in patterns]
    txts = [bytes(t) for t in texts]
    po = np.zeros(len(pats) + 1, np.uint64)
    po[1:] = np.cumsum([len(p) for p in pats])
    to = np.zeros(len(txts) + 1, np.uint64)
    to[1:] = np.cumsum([len(t) for t in txts])
    P = np.frombuffer(b"".join(pats), np.uint8).copy()
    T = np.frombuffer(b"".join(txts), np.uint8).copy()
    out = np.empty(max(int(to[-1]), 1), np.int32)
    _check(load().peanut_debug_bitvector_columns(P.ctypes.data, po.ctypes.data, len(pats), T.ctypes.data,
                                                 to.ctypes.data, out.ctypes.data, _stream_ptr(stream)))
    return [out[int(to[i]):int(to[i + 1])].copy() for i in range(len(pats))]


def bitvector_columns_noalloc(d_pat, d_pat_off, d_txt, d_txt_off, d_out, stream=None):
    """peanut_bitvector_columns_noalloc: the same columns with every buffer in device memory
    (torch tensors: uint8 patterns / texts, int64 offsets, int32 output) and no allocation
    inside the library; its scratch is a fixed array of up to 8192 patterns' masks."""
    _check(load().peanut_bitvector_columns_noalloc(d_pat.data_ptr(), d_pat_off.data_ptr(), int(d_pat_off.numel()) - 1,
                                                   d_txt.data_ptr(), d_txt_off.data_ptr(), d_out.data_ptr(),
                                                   _stream_ptr(stream)))


# ---- batched and served mapping ------------------------------------------------------------

TIMEOUT = 4  # peanut_status PEANUT_TIMEOUT
RESULT_ON_DEVICE = 0x100  # PEANUT_RESULT_ON_DEVICE


class Engine(_Handle):
    """peanut_engine: submissions of any size and length mix, coalesced into per-q-class launches
    on `executors` concurrent streams, admitted by a device-memory budget.  Inputs passed to
    submit() are kept referenced here until their result is taken with wait()."""

    def __init__(self, ref: Reference, k=None, k_permille=None, executors: int = 2, max_reads: int = 0,
                 autotune: bool = True, fixed_q: int = 0, hbm_budget: int = 0, graphs: bool = False):
        if k is None and k_permille is None:
            raise ValueError("give k or k_permille")
        p = EngineParams(K_FROM_PERMILLE if k is None else int(k), int(k_permille or 0), int(executors),
                         int(max_reads), int(bool(autotune)), int(fixed_q), int(hbm_budget), int(bool(graphs)))
        out = c_void_p()
        _check(load().peanut_engine_create(ref.ptr, ctypes.byref(p), ctypes.byref(out)))
        super().__init__(out.value)
        self.ref = ref
        self._inputs = {}

    def submit(self, seq, offsets, mode: str = "all") -> int:
        """peanut_engine_submit: host reads; returns the ticket."""
        s = _host_u8(seq)
        o = np.ascontiguousarray(offsets, dtype=np.uint64)
        t = c_uint64()
        _check(load().peanut_engine_submit(self.ptr, s.ctypes.data, o.ctypes.data, o.size - 1, MODES[mode],
                                           ctypes.byref(t)))
        self._inputs[t.value] = (s, o)
        return int(t.value)

    def submit_device(self, d_seq, d_offsets, mode: str = "all", result_on_device: bool = False) -> int:
        """peanut_engine_submit_device: reads in device memory (torch uint8 / int64 tensors, writes
        complete); with result_on_device the hits stay on the device (wait_device)."""
        t = c_uint64()
        flags = RESULT_ON_DEVICE if result_on_device else 0
        _check(load().peanut_engine_submit_device(self.ptr, d_seq.data_ptr(), d_offsets.data_ptr(),
                                                  int(d_offsets.numel()) - 1, int(d_seq.numel()),
                                                  MODES[mode] | flags, ctypes.byref(t)))
        self._inputs[t.value] = (d_seq, d_offsets)
        return int(t.value)

    def wait_arrays(self, ticket: int, timeout_ms: int = -1) -> HostHits | None:
        """peanut_engine_wait: the submission's hits as library-held numpy views, or None on
        timeout."""
        hp = POINTER(Hits)()
        st = load().peanut_engine_wait(self.ptr, int(ticket), int(timeout_ms), ctypes.byref(hp))
        if st == TIMEOUT:
            return None
        self._inputs.pop(int(ticket), None)
        _check(st)
        return HostHits(hp)

    def wait(self, ticket: int, timeout_ms: int = -1) -> np.ndarray | None:
        """peanut_engine_wait: the submission's hit set (structured array), or None on timeout."""
        h = self.wait_arrays(ticket, timeout_ms)
        if h is None:
            return None
        try:
            out = np.empty(h.n, HIT_DTYPE)
            out["read"] = h.read
            out["strand"] = h.strand
            out["end"] = h.end.astype(np.int64)
            out["dist"] = h.dist
            return out
        finally:
            h.free()

    def wait_device(self, ticket: int, timeout_ms: int = -1) -> DeviceHits | None:
        """peanut_engine_wait_device: the submission's hits left in device memory, or None on
        timeout."""
        hp = POINTER(DeviceHitsStruct)()
        st = load().peanut_engine_wait_device(self.ptr, int(ticket), int(timeout_ms), ctypes.byref(hp))
        if st == TIMEOUT:
            return None
        self._inputs.pop(int(ticket), None)
        _check(st)
        return DeviceHits(hp)

    def stats(self) -> dict:
        s = EngineStats()
        _check(load().peanut_engine_get_stats(self.ptr, ctypes.byref(s)))
        d = {f: getattr(s, f) for f, _ in EngineStats._fields_ if f != "cls"}
        d["classes"] = [{f: getattr(s.cls[i], f) for f, _ in EngineClass._fields_} for i in range(s.n_classes)]
        return d

    def free(self):
        super().free()
        self._inputs = {}
