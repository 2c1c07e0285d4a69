"""CPU-side checks of the C ABI: the library builds, loads and exports every declared symbol,
and argument errors come back as status codes (no GPU needed for these)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "peanut.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(peanut_[a-z_]+)\s*\(", src)) - {"peanut_alloc_fn", "peanut_release_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_1403_1706_gb300 import build, peanut
    build.build()
    return peanut.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("peanut_pack_reference", "peanut_index_reads", "peanut_map", "peanut_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_argument_errors_are_status_codes(lib):
    from paper_1403_1706_gb300 import peanut
    out = ctypes.c_void_p()
    # NULL sequence
    assert lib.peanut_pack_reference(None, 10, None, ctypes.byref(out)) == 1
    assert b"NULL" in lib.peanut_last_error()
    # q out of range is rejected before any device work
    p = peanut.Params(17, 5, 0, 0, None)
    fake = ctypes.c_void_p()
    st = lib.peanut_index_reads(None, b"ACGT", (ctypes.c_uint64 * 2)(0, 4), 1, ctypes.byref(p), ctypes.byref(fake))
    assert st == 1  # bad reference checked first
    # freeing NULL is a no-op
    lib.peanut_free(None)
    # a mismatched allocator pair is refused
    assert lib.peanut_set_allocator(peanut.ALLOC_FN(lambda a, b, c: None), peanut.RELEASE_FN(), None) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1403_1706_gb300 import peanut
    monkeypatch.setattr(peanut, "_lib", None)
    monkeypatch.setattr(peanut, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        peanut.load()
