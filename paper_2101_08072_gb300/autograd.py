"""torch.autograd wrapper of the measurement operator R.

forward:  V = R x (pfb_degrid), x real [nband, nx, ny] -> V complex [nrow, nchan].
backward: with PyTorch's convention for a real loss L of a complex tensor
(grad = dL/dRe V + i dL/dIm V), dL/dx_p = Re sum_k conj(R_kp) grad_k = (R^dagger grad)_p,
i.e. the gridding adjoint with unit weights (pfb_grid), exactly the transpose the
library implements.  For f(x) = 1/2 (V - Rx)^dagger Sigma^-1 (V - Rx) (Eq. 2) this
gives the gradient -R^dagger Sigma^-1 (V - Rx) of Eq. 3.
"""
from __future__ import annotations

import torch

from .ops import Context, Geometry, default_context


class DegridFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x, geom: Geometry, uvw, freq, band_of_chan, pctx: Context):
        fctx.geom = geom
        fctx.pctx = pctx
        fctx.save_for_backward(uvw, freq, band_of_chan)
        return pctx.pfb_degrid(geom, uvw, freq, band_of_chan, x.contiguous())

    @staticmethod
    def backward(fctx, grad_v):
        uvw, freq, band_of_chan = fctx.saved_tensors
        gx = fctx.pctx.pfb_grid(fctx.geom, uvw, freq, band_of_chan, grad_v.contiguous())
        return gx, None, None, None, None, None


def degrid(x, geom: Geometry, uvw, freq, band_of_chan, pctx: Context | None = None):
    """Differentiable R x."""
    return DegridFn.apply(x, geom, uvw, freq, band_of_chan, pctx or default_context(x.device.index))


def data_fidelity(x, vis, wgt, geom: Geometry, uvw, freq, band_of_chan, pctx: Context | None = None):
    """f(x) = 1/2 (V - Rx)^dagger Sigma^-1 (V - Rx) (Eq. 2), accumulated in FP64."""
    r = vis - degrid(x, geom, uvw, freq, band_of_chan, pctx)
    return 0.5 * (wgt.double() * (r.real.double() ** 2 + r.imag.double() ** 2)).sum()
