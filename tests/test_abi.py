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
