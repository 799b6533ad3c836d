"""The C-ABI library loads on the host and exports every function that
include/nmf_gb300.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nmf_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(nmf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    builder = __graft_entry__._load_builder()
    path = builder.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("nmf_init", "nmf_iterate", "nmf_nls_bpp", "nmf_objective", "nmf_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.nmf_status_str.restype = ctypes.c_char_p
    assert lib.nmf_status_str(0) == b"NMF_OK"
    assert lib.nmf_status_str(4) == b"NMF_ERR_NOT_CONVERGED"


def test_invalid_arguments_rejected_before_launch(lib):
    # Host-side validation: these return INVALID_ARG without touching a GPU.
    lib.nmf_gram.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                             ctypes.c_void_p]
    assert lib.nmf_gram(None, 10, 0, None, None) == 1          # k = 0
    assert lib.nmf_gram(None, 10, 129, None, None) == 1        # k > NMF_MAX_K
    lib.nmf_nls_bpp.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.nmf_nls_bpp(None, None) == 1                    # null descriptor
    lib.nmf_init.argtypes = [ctypes.c_void_p] * 6
    assert lib.nmf_init(None, None, None, None, None, None) == 1


def test_python_binding_exports_same_names():
    src = open(os.path.join(ROOT, "paper_1509_09313_gb300", "__init__.py")).read()
    for n in declared_functions():
        assert n in src, n


def test_launch_shape_set_and_get(lib):
    # Host-only state: the shape later solves of k use.
    I = ctypes.c_int32
    lib.nmf_nls_bpp_set_shape.argtypes = [I, I, I, I]
    lib.nmf_nls_bpp_get_shape.argtypes = [I] + [ctypes.POINTER(I)] * 3
    w, c, g = I(0), I(0), I(0)
    assert lib.nmf_nls_bpp_get_shape(50, ctypes.byref(w), ctypes.byref(c), ctypes.byref(g)) == 0
    # The default: group pass on the SIMT pipes, on the tensor cores for
    # 65 <= k <= 112.
    assert (w.value, c.value, g.value) == (8, 8, 1)
    for kk, gg in ((64, 1), (65, 2), (100, 2), (112, 2), (113, 1), (128, 1)):
        assert lib.nmf_nls_bpp_get_shape(kk, ctypes.byref(w), ctypes.byref(c), ctypes.byref(g)) == 0
        assert (w.value, c.value, g.value) == (8, 8, gg), kk
    assert lib.nmf_nls_bpp_set_shape(50, 16, 4, 0) == 0
    lib.nmf_nls_bpp_get_shape(50, ctypes.byref(w), ctypes.byref(c), ctypes.byref(g))
    assert (w.value, c.value, g.value) == (16, 4, 0)
    assert lib.nmf_nls_bpp_set_shape(50, 8, 8, 1) == 0
    for bad in [(0, 8, 8, 1), (129, 8, 8, 1), (50, 0, 8, 1), (50, 17, 8, 1),
                (50, 8, 0, 1), (50, 8, 1025, 1), (50, 8, 8, 3), (50, 8, 8, -1),
                (113, 8, 8, 2)]:
        assert lib.nmf_nls_bpp_set_shape(*bad) == 1, bad
    assert lib.nmf_nls_bpp_get_shape(0, None, None, None) == 1
    assert lib.nmf_nls_bpp_set_shape(50, 8, 8, 2) == 0
    assert lib.nmf_nls_bpp_set_shape(50, 8, 8, 1) == 0


class NlsDesc(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("nrhs", ctypes.c_int64), ("G", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("X", ctypes.c_void_p), ("passive_in", ctypes.c_void_p),
                ("passive_out", ctypes.c_void_p), ("rounds_out", ctypes.c_void_p),
                ("status_out", ctypes.c_void_p), ("max_rounds", ctypes.c_int32)]


@pytest.mark.parametrize("fn", ["nmf_nls_bpp", "nmf_nls_bpp_noalloc"])
def test_nls_rejects_overlapping_x_and_b(lib, fn):
    # X must not overlap B: checked on the host before anything is launched
    # (the pointers below are never dereferenced).
    f = getattr(lib, fn)
    f.argtypes = [ctypes.POINTER(NlsDesc), ctypes.c_void_p]
    k, nrhs = 10, 100
    for x_off in (0, 4 * k * nrhs - 4, -(4 * k * nrhs - 4)):
        d = NlsDesc(k, nrhs, 0x10000, 0x200000, 0x200000 + x_off, None, None, None, None, 10)
        assert f(ctypes.byref(d), None) == 1, x_off


def test_struct_layouts_match_header(tmp_path):
    # The binding's ctypes structures mirror the header's: same size and the
    # same offset for every field (compiled against the header with gcc).
    import subprocess

    import paper_1509_09313_gb300 as lib
    names = ["nmf_config", "nmf_matrix", "nmf_nls_desc", "nmf_stats"]
    lines = ['#include <stdio.h>', '#include "nmf_gb300.h"', "int main(void) {"]
    for s in names:
        lines.append(f'    printf("{s} %zu\\n", sizeof({s}));')
        for f in getattr(lib, s)._fields_:
            lines.append(f'    printf("{s}.{f[0]} %zu\\n", offsetof({s}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    c_side = dict(line.split() for line in out.splitlines())
    for s in names:
        st = getattr(lib, s)
        assert int(c_side[s]) == ctypes.sizeof(st), s
        for f in st._fields_:
            assert int(c_side[f"{s}.{f[0]}"]) == getattr(st, f[0]).offset, (s, f[0])
