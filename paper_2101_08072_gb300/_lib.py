"""ctypes declarations of libpfb's C ABI (include/pfb.h)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpfb.so")

PFB_F32 = 0
PFB_F64 = 1
PFB_NO_DIVIDE_BY_N = 1
PFB_NO_WTERM = 2
PFB_NO_ITEM_RECORDS = 4
PFB_ACCUMULATE = 8
PFB_NO_PRUNED_FFT = 16
PFB_STEP_APPROX_GRADIENT = 1
PFB_STEP_SAFE_GAMMA = 2
PFB_SAFE_GAMMA_ITERS = 30

ERRORS = {
    0: "PFB_OK", -1: "PFB_ERR_ARG", -2: "PFB_ERR_OOM", -3: "PFB_ERR_CUDA", -4: "PFB_ERR_EPS",
    -5: "PFB_ERR_TIMEOUT", -6: "PFB_ERR_NOT_IMPLEMENTED",
}

# every function the header declares (the CPU test checks the library exports them)
EXPORTS = ["pfb_create", "pfb_destroy", "pfb_last_error", "pfb_plan_reset", "pfb_degrid", "pfb_grid",
           "pfb_dirty", "pfb_psf", "pfb_hessian", "pfb_hessian_host", "pfb_psf_conv", "pfb_step", "pfb_clean",
           "pfb_version",
           "pfb_timing", "pfb_timing_read", "pfb_timing_names", "pfb_wsum_static", "pfb_kernel_support",
           "pfb_step_bound", "pfb_last_step_bound"]


class pfb_geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dl", ctypes.c_double),
                ("dm", ctypes.c_double), ("fov_l", ctypes.c_double), ("fov_m", ctypes.c_double),
                ("epsilon", ctypes.c_double), ("nband", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("l0", ctypes.c_double), ("m0", ctypes.c_double)]


class pfb_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("sigma", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("cg_tol", ctypes.c_double), ("pd_tol", ctypes.c_double), ("cg_iters", ctypes.c_int32),
                ("pd_iters", ctypes.c_int32), ("nlevel", ctypes.c_int32), ("basis_mask", ctypes.c_uint32),
                ("unorm", ctypes.c_double), ("flags", ctypes.c_uint32)]


class PfbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libpfb.so.  There is no fallback: a missing library is an error."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpfb.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    G = ctypes.POINTER(pfb_geom)
    lib.pfb_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t]
    lib.pfb_create.restype = ctypes.c_int
    lib.pfb_destroy.argtypes = [P]
    lib.pfb_destroy.restype = None
    lib.pfb_last_error.argtypes = [P]
    lib.pfb_last_error.restype = ctypes.c_char_p
    lib.pfb_plan_reset.argtypes = [P]
    lib.pfb_version.restype = ctypes.c_char_p
    data = [I64, I32, P, P, P]
    lib.pfb_degrid.argtypes = [P, G, ctypes.c_int, *data, P, P, P]
    lib.pfb_grid.argtypes = [P, G, ctypes.c_int, *data, P, P, P, P]
    lib.pfb_dirty.argtypes = [P, G, ctypes.c_int, *data, P, P, P, ctypes.POINTER(D), P]
    lib.pfb_psf.argtypes = [P, G, ctypes.c_int, *data, P, P, ctypes.POINTER(D), P]
    lib.pfb_hessian.argtypes = [P, G, ctypes.c_int, *data, P, P, P, P]
    lib.pfb_hessian_host.argtypes = [P, G, ctypes.c_int, *data, P, P, P, P]
    lib.pfb_psf_conv.argtypes = [P, G, ctypes.c_int, P, P, P, P]
    lib.pfb_step.argtypes = [P, G, ctypes.c_int, ctypes.POINTER(pfb_params), *data, P, P, P,
                             ctypes.POINTER(D), P, P, ctypes.POINTER(I64), ctypes.POINTER(D), P]
    lib.pfb_clean.argtypes = [P, G, ctypes.c_int, ctypes.POINTER(pfb_params), I32, D, *data, P, P, P, P,
                              ctypes.POINTER(D), P, P, ctypes.POINTER(I32), ctypes.POINTER(I64),
                              ctypes.POINTER(D), P]
    lib.pfb_step_bound.argtypes = [P, G, ctypes.c_int, ctypes.POINTER(pfb_params), *data, P, P,
                                   ctypes.POINTER(D), P, I32, ctypes.POINTER(D), P]
    lib.pfb_last_step_bound.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.pfb_timing.argtypes = [P, ctypes.c_int]
    lib.pfb_timing_read.argtypes = [P, ctypes.c_char_p, ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.pfb_timing_names.argtypes = [P, ctypes.c_char_p, ctypes.c_size_t]
    lib.pfb_wsum_static.argtypes = [ctypes.c_int, ctypes.c_int, I64, I32, I32, P, P, P, P]
    lib.pfb_kernel_support.argtypes = [D, ctypes.c_int]
    for f in EXPORTS:
        if f not in ("pfb_destroy", "pfb_last_error", "pfb_version", "pfb_create"):
            getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib
