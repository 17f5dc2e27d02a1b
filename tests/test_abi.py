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


def test_struct_layouts_match_header(tmp_path):
    """Sizes and field offsets of the ctypes structs against the C compiler's view of
    include/pfb.h."""
    import shutil
    import subprocess
    from paper_2101_08072_gb300 import _lib
    assert ctypes.sizeof(_lib.pfb_geom) == 72
    assert ctypes.sizeof(_lib.pfb_params) == 72
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pfb.h"', 'int main(void) {']
    for st in (_lib.pfb_geom, _lib.pfb_params):
        cname = st.__name__
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in st._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {cf}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in (_lib.pfb_geom, _lib.pfb_params):
        assert got[(st.__name__, "size")] == ctypes.sizeof(st)
        for f, _ in st._fields_:
            assert got[(st.__name__, f)] == getattr(st, f).offset, (st.__name__, f)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2101_08072_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def _es_hat(W, beta, xi):
    """Fourier transform of the ES kernel exp(beta (sqrt(1 - (2z/W)^2) - 1)) on |z| < W/2,
    by adaptive quadrature in z (independent of the library's Gauss-Legendre rule in
    the sine-substituted variable)."""
    import warnings
    import numpy as np
    from scipy.integrate import IntegrationWarning, quad
    f = lambda z: np.exp(beta * (np.sqrt(max(0.0, 1.0 - (2.0 * z / W) ** 2)) - 1.0)) * np.cos(2 * np.pi * xi * z)
    with warnings.catch_warnings():
        # the alias terms are 1e-5..1e-12 of hat(0): a few correct digits of them suffice
        warnings.simplefilter("ignore", IntegrationWarning)
        return 2.0 * quad(f, 0.0, W / 2.0, limit=200, epsabs=1e-16, epsrel=1e-13)[0]


def _alias_bound(W):
    """min over beta in {2.0, 2.05, ..., 2.4} W of max_{|xi| <= 1/4} sum_{m=+-1,+-2} |hat(xi+m)| / hat(xi):
    the aliasing error of 2x-oversampled gridding with the ES kernel (Section 2)."""
    best = float("inf")
    for k in range(9):
        beta = (2.0 + 0.05 * k) * W
        worst = 0.0
        for i in range(26):
            xi = 0.25 * i / 25.0
            a = sum(abs(_es_hat(W, beta, xi + m)) for m in (-2, -1, 1, 2))
            worst = max(worst, a / _es_hat(W, beta, xi))
        best = min(best, worst)
    return best


def test_kernel_support_follows_the_aliasing_bound(lib):
    """pfb_kernel_support(eps) is the smallest W whose aliasing bound is <= eps: checked
    just above and just below the bound of each W, recomputed here from the kernel."""
    lib.pfb_kernel_support.argtypes = [ctypes.c_double, ctypes.c_int]
    lib.pfb_kernel_support.restype = ctypes.c_int
    F32, F64 = 0, 1
    bounds = {W: _alias_bound(W) for W in range(4, 12)}
    assert all(bounds[W + 1] < bounds[W] for W in range(4, 11))   # more taps, smaller error
    for W in range(5, 12):
        prec = F32 if bounds[W] * 1.05 >= 1e-6 else F64
        assert lib.pfb_kernel_support(bounds[W] * 1.05, prec) == W, W
        if bounds[W] * 0.95 >= (1e-6 if prec == F32 else 1e-12):
            assert lib.pfb_kernel_support(bounds[W] * 0.95, prec) == W + 1, W
    # the FP32 path's working point (eps = 3e-5) takes W = 6
    assert lib.pfb_kernel_support(3e-5, F32) == 6
    # errors: not positive / not finite -> PFB_ERR_ARG; beyond the precision -> PFB_ERR_EPS
    assert lib.pfb_kernel_support(0.0, F32) == -1
    assert lib.pfb_kernel_support(float("nan"), F32) == -1
    assert lib.pfb_kernel_support(1e-7, F32) == -4
    assert lib.pfb_kernel_support(1e-13, F64) == -4
    assert lib.pfb_kernel_support(1e-3, 7) == -1
