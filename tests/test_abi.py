"""The C ABI library builds, loads and exports every entry point include/vie.h declares (no GPU needed)."""
import ctypes
import os
import re

from paper_2501_13512_gb300 import build, vie


def test_library_builds_and_exports_header_symbols():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = vie.declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert lib.vie_version() == 100


def test_header_documents_every_entry_point():
    text = open(vie.HEADER).read()
    for name in vie.declared_functions():
        # each declaration is preceded by a comment block
        i = re.search(r"^\s*int\s+" + name + r"\s*\(", text, re.M).start()
        assert "*/" in text[max(0, i - 1500):i], name


def test_error_text_roundtrip_without_gpu():
    lib = vie.load()
    # a null descriptor is rejected before any CUDA call
    rc = lib.vie_grid_create(None, None)
    assert rc == vie.VIE_EINVAL
    assert "null" in vie.last_error()


def test_struct_sizes_match_header_layout():
    # field order and widths of the public structs, as laid out by the C compiler
    assert ctypes.sizeof(vie.GridDesc) == 4 * 3 + 4 + 8 + 8 + 8 + 8
    assert ctypes.sizeof(vie.SolveOpts) == 8 + 8 + 4 * 5 + 4 + 8
    assert ctypes.sizeof(vie.PrecondStats) == 4 + 4 + 8 + 4 + 4
