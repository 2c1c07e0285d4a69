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
    p = peanut.Params(q=17, k_fixed=5)
    fake = ctypes.c_void_p()
    st = lib.peanut_index_reads(None, b"ACGT", (ctypes.c_uint64 * 2)(0, 4), 1, ctypes.byref(p), ctypes.byref(fake))
    assert st == 1  # bad reference checked first
    # freeing NULL is a no-op
    lib.peanut_free(None)
    # a mismatched allocator pair is refused
    assert lib.peanut_set_allocator(peanut.ALLOC_FN(lambda a, b, c: None), peanut.RELEASE_FN(), None) == 1


def test_engine_argument_errors(lib):
    from paper_1403_1706_gb300 import peanut
    out = ctypes.c_void_p()
    p = peanut.EngineParams(k_fixed=5)
    assert lib.peanut_engine_create(None, ctypes.byref(p), ctypes.byref(out)) == 1
    t = ctypes.c_uint64()
    assert lib.peanut_engine_submit(None, b"ACGT", (ctypes.c_uint64 * 2)(0, 4), 1, 0, ctypes.byref(t)) == 1
    hp = ctypes.POINTER(peanut.Hits)()
    assert lib.peanut_engine_wait(None, 1, 0, ctypes.byref(hp)) == 1


STRUCTS = {"peanut_params": "Params", "peanut_map_stats": "MapStats", "peanut_hits": "Hits",
           "peanut_device_hits": "DeviceHitsStruct", "peanut_engine_params": "EngineParams",
           "peanut_engine_class": "EngineClass", "peanut_engine_stats": "EngineStats"}


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the C header's size and field offsets."""
    import shutil
    import subprocess
    from paper_1403_1706_gb300 import peanut
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = []
    for cname, pname in STRUCTS.items():
        cls = getattr(peanut, pname)
        lines.append(f'printf("{pname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{pname} {f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"peanut.h\"\nint main(void){"
                   + "".join(lines) + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, got):
        pname, field, val = line.split()
        cls = getattr(peanut, pname)
        want = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert int(val) == want, (pname, field)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1403_1706_gb300 import peanut
    monkeypatch.setattr(peanut, "_lib", None)
    monkeypatch.setattr(peanut, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        peanut.load()
