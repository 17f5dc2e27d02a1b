"""GB300 (sm_103a) implementation of the pfb-clean hot path: the wide-field
measurement operator R, its weighted adjoint, the dirty image, the PSF, the
exact Hessian-vector product, the PSF convolution and one preconditioned
forward-backward step, behind the C ABI of include/pfb.h (libpfb.so).

The binding loads libpfb.so on first use and has no fallback: without the
built library every entry point raises.
"""
from ._lib import PFB_F32, PFB_F64, PFB_NO_DIVIDE_BY_N, PFB_NO_WTERM, PfbError  # noqa: F401

__all__ = ["Context", "Geometry", "StepParams", "default_context", "version", "PfbError",
           "PFB_F32", "PFB_F64", "PFB_NO_DIVIDE_BY_N", "PFB_NO_WTERM"]


def __getattr__(name):
    # torch-dependent parts load lazily so that `synth` imports without torch/CUDA
    if name in ("Context", "Geometry", "StepParams", "default_context", "version"):
        from . import ops
        return getattr(ops, name)
    raise AttributeError(name)
