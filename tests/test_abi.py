"""The C ABI library builds, loads and exports every entry point include/vie.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np

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


STRUCTS = {"vie_grid_desc": "GridDesc", "vie_grid_info": "GridInfo", "vie_precond_stats": "PrecondStats",
           "vie_solve_opts": "SolveOpts", "vie_solve_stats": "SolveStats", "vie_batch_desc": "BatchDesc",
           "vie_kernel_stat": "KernelStat"}


def test_struct_layouts_match_header(tmp_path):
    # every field offset and struct size of the ctypes binding, against the C compiler's layout of include/vie.h
    lines = ["#include <stddef.h>", "#include <stdio.h>", f'#include "{vie.HEADER}"', "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        cls = getattr(vie, pyname)
        lines.append(f'printf("{pyname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{pyname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    for pyname in STRUCTS.values():
        cls = getattr(vie, pyname)
        assert got[(pyname, "size")] == ctypes.sizeof(cls), pyname
        for field, _ in cls._fields_:
            assert got[(pyname, field)] == getattr(cls, field).offset, (pyname, field)


def test_argument_validation_without_gpu():
    # limits and malformed arguments are rejected before any CUDA call, with a message
    lib = vie.load()
    eps = np.ones(2 * 4, dtype=np.float64)
    for dims, h in (((513, 1, 1), 1.0), ((0, 4, 1), 1.0), ((2, 2, 1), 0.0), ((2, 2, 1), float("nan"))):
        d = vie.GridDesc(dims[0], dims[1], dims[2], h, eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0)
        out = ctypes.c_void_p()
        assert lib.vie_grid_create(ctypes.byref(d), ctypes.byref(out)) == vie.VIE_EINVAL, (dims, h)
        assert out.value is None
        assert vie.last_error()
    d = vie.GridDesc(2, 2, 1, 1.0, eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 7)
    assert lib.vie_grid_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == vie.VIE_EINVAL
    for expand in (-1, 65):
        d = vie.GridDesc(2, 2, 1, 1.0, eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0, expand)
        assert lib.vie_grid_create(ctypes.byref(d), ctypes.byref(ctypes.c_void_p())) == vie.VIE_EINVAL
        assert "block_expand" in vie.last_error()
    for count in (0, 21846):
        b = vie.BatchDesc(2, 2, 1, 1.0, count, eps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
        assert lib.vie_batch_create(ctypes.byref(b), ctypes.byref(ctypes.c_void_p())) == vie.VIE_EINVAL
    # the no-allocation MVM: padded volume above 32768 points (17^3 pads to 64^3), null pointers
    buf = ctypes.c_void_p(16)
    assert lib.vie_matvec_noalloc(17, 17, 17, 1.0, 1.0, buf, buf, buf, None) == vie.VIE_EINVAL
    assert "exceeds" in vie.last_error()
    assert lib.vie_matvec_noalloc(4, 4, 4, 1.0, 1.0, None, buf, buf, None) == vie.VIE_EINVAL


def test_python_binding_exposes_every_public_wrapper():
    # the ctypes binding's public wrappers of the merge-session, batch and host-buffer entry points exist
    from paper_2501_13512_gb300 import vie
    for name in ("Grid", "Spectrum", "Batch", "Rooftop", "MergeSession", "solve_many", "batch_solve_many"):
        assert hasattr(vie, name), name
    for meth in ("solve", "solve_host", "precond", "matvec", "spectrum", "plane_wave", "far_field_rcs"):
        assert hasattr(vie.Grid, meth), meth
