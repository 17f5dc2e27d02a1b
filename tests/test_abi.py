"""CPU checks of the boundary: the library builds for sm_103a, loads, and exports
every entry point that include/pfb.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import _lib
    return ctypes.CDLL(_lib.LIB_PATH)


def header_functions():
    src = open(os.path.join(ROOT, "include", "pfb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pfb_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    fns = header_functions()
    for f in ("pfb_degrid", "pfb_grid", "pfb_dirty", "pfb_psf", "pfb_hessian", "pfb_psf_conv", "pfb_step"):
        assert f in fns


def test_library_exports_every_declared_symbol(lib):
    from paper_2101_08072_gb300 import _lib
    for f in header_functions():
        assert hasattr(lib, f), f
    assert sorted(_lib.EXPORTS) == header_functions()


def test_version_and_no_device(lib):
    lib.pfb_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.pfb_version()
    import torch
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        lib.pfb_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]
        assert lib.pfb_create(ctypes.byref(h), 0, 0) == -1   # no device: argument error, no crash


def test_struct_layouts_match_header():
    from paper_2101_08072_gb300 import _lib
    assert ctypes.sizeof(_lib.pfb_geom) == 56
    assert ctypes.sizeof(_lib.pfb_params) == 64


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2101_08072_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved
