"""Python binding of libpfb: the entry points of include/pfb.h, same names, on
torch tensors.  Argument marshalling only (shapes, dtypes, device pointers,
the current CUDA stream); every step of the computation runs in libpfb's
kernels.  Tensors must be contiguous and on the context's device.

Precision follows the dtype: float32 images / complex64 visibilities select
PFB_F32 (FP64 coordinates and phases inside), float64 / complex128 select PFB_F64.
"""
from __future__ import annotations

import ctypes
import dataclasses
import threading

import numpy as np
import torch

from . import _lib
from ._lib import PFB_F32, PFB_F64, PfbError


@dataclasses.dataclass
class Geometry:
    """Image geometry and accuracy (pfb_geom)."""
    nx: int
    ny: int
    dl: float
    dm: float
    nband: int = 1
    epsilon: float = 1e-5
    flags: int = 0
    l0: float = 0.0   # direction cosines of the image centre: a facet of a wider field
    m0: float = 0.0

    def c(self) -> _lib.pfb_geom:
        return _lib.pfb_geom(self.nx, self.ny, self.dl, self.dm, 0.0, 0.0, self.epsilon, self.nband, self.flags,
                             self.l0, self.m0)


@dataclasses.dataclass
class StepParams:
    """Parameters of one pfb-clean step (pfb_params)."""
    gamma: float = 1.0
    sigma: float = 1e-3
    lam: float = 1e-4
    cg_tol: float = 0.0
    pd_tol: float = 0.0
    cg_iters: int = 50
    pd_iters: int = 100
    nlevel: int = 3
    basis_mask: int = 1
    unorm: float = 0.0
    approx_gradient: bool = False   # Eq. 4 (I^psf * x) in place of the Hessian (PFB_STEP_APPROX_GRADIENT)
    safe_gamma: bool = False        # pfb_clean: gamma capped at 1.9 / lambda_max(U^-1 H) (PFB_STEP_SAFE_GAMMA)

    def c(self) -> _lib.pfb_params:
        flags = (_lib.PFB_STEP_APPROX_GRADIENT if self.approx_gradient else 0) | \
                (_lib.PFB_STEP_SAFE_GAMMA if self.safe_gamma else 0)
        return _lib.pfb_params(self.gamma, self.sigma, self.lam, self.cg_tol, self.pd_tol, self.cg_iters,
                               self.pd_iters, self.nlevel, self.basis_mask, self.unorm, flags)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _prec_real(dtype) -> int:
    if dtype == torch.float32:
        return PFB_F32
    if dtype == torch.float64:
        return PFB_F64
    raise TypeError(f"image dtype must be float32 or float64, got {dtype}")


def _prec_cx(dtype) -> int:
    if dtype == torch.complex64:
        return PFB_F32
    if dtype == torch.complex128:
        return PFB_F64
    raise TypeError(f"visibility dtype must be complex64 or complex128, got {dtype}")


_RDT = {PFB_F32: torch.float32, PFB_F64: torch.float64}
_CDT = {PFB_F32: torch.complex64, PFB_F64: torch.complex128}


class Context:
    """A libpfb context on one CUDA device (plans, scratch, cuFFT handles)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.lib = _lib.load()
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        rc = self.lib.pfb_create(ctypes.byref(h), device, hbm_budget_bytes)
        if rc != 0:
            raise PfbError(rc, f"pfb_create(device={device}) failed")
        self.h = h
        # Inputs of the plans cached by libpfb, most recent last.  libpfb keys its
        # plans on device pointers; holding the tensors keeps torch's caching
        # allocator from handing the same addresses to different data while a plan
        # that points at them may still be cached (libpfb keeps at most 16 plans).
        self._keep: list[tuple] = []

    def close(self):
        if getattr(self, "h", None):
            self.lib.pfb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ helpers
    def _check(self, rc: int):
        if rc != 0:
            raise PfbError(rc, self.lib.pfb_last_error(self.h).decode())

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _data(self, uvw, freq, band_of_chan):
        for name, t, dt in (("uvw", uvw, torch.float64), ("freq", freq, torch.float64),
                            ("band_of_chan", band_of_chan, torch.int32)):
            if t.dtype != dt or not t.is_contiguous() or t.device != self.device:
                raise TypeError(f"{name} must be a contiguous {dt} tensor on {self.device}")
        if uvw.ndim != 2 or uvw.shape[1] != 3:
            raise ValueError("uvw must be [nrow, 3]")
        key = (uvw.data_ptr(), freq.data_ptr(), band_of_chan.data_ptr())
        self._keep = [k for k in self._keep if k[0] != key] + [(key, uvw, freq, band_of_chan)]
        del self._keep[:-16]
        return uvw.shape[0], freq.shape[0]

    def _t(self, t, name, dtype, shape):
        if t.dtype != dtype or not t.is_contiguous() or t.device != self.device or tuple(t.shape) != tuple(shape):
            raise TypeError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)} on {self.device}")
        return t

    # ------------------------------------------------------------------ entry points
    def pfb_degrid(self, geom: Geometry, uvw, freq, band_of_chan, image, out=None):
        """R x (Eq. 1): image [nband, nx, ny] -> visibilities [nrow, nchan]."""
        nrow, nchan = self._data(uvw, freq, band_of_chan)
        prec = _prec_real(image.dtype)
        self._t(image, "image", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        if out is None:
            out = torch.empty((nrow, nchan), dtype=_CDT[prec], device=self.device)
        self._t(out, "vis_out", _CDT[prec], (nrow, nchan))
        g = geom.c()
        self._check(self.lib.pfb_degrid(self.h, ctypes.byref(g), prec, nrow, nchan, _ptr(uvw), _ptr(freq),
                                        _ptr(band_of_chan), _ptr(image), _ptr(out), self._stream()))
        return out

    def pfb_grid(self, geom: Geometry, uvw, freq, band_of_chan, vis, wgt=None, out=None):
        """R^dagger Sigma^-1 y (Eq. 3): visibilities -> image [nband, nx, ny]."""
        nrow, nchan = self._data(uvw, freq, band_of_chan)
        prec = _prec_cx(vis.dtype)
        self._t(vis, "vis", _CDT[prec], (nrow, nchan))
        if wgt is not None:
            self._t(wgt, "wgt", _RDT[prec], (nrow, nchan))
        if out is None:
            out = torch.empty((geom.nband, geom.nx, geom.ny), dtype=_RDT[prec], device=self.device)
        self._t(out, "image_out", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        g = geom.c()
        self._check(self.lib.pfb_grid(self.h, ctypes.byref(g), prec, nrow, nchan, _ptr(uvw), _ptr(freq),
                                      _ptr(band_of_chan), _ptr(vis), _ptr(wgt), _ptr(out), self._stream()))
        return out

    def pfb_dirty(self, geom: Geometry, uvw, freq, band_of_chan, vis, wgt=None, out=None):
        """I^d = R^dagger Sigma^-1 V and the per-band weight sums (numpy, host)."""
        nrow, nchan = self._data(uvw, freq, band_of_chan)
        prec = _prec_cx(vis.dtype)
        self._t(vis, "vis", _CDT[prec], (nrow, nchan))
        if wgt is not None:
            self._t(wgt, "wgt", _RDT[prec], (nrow, nchan))
        if out is None:
            out = torch.empty((geom.nband, geom.nx, geom.ny), dtype=_RDT[prec], device=self.device)
        self._t(out, "image_out", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        ws = (ctypes.c_double * geom.nband)()
        g = geom.c()
        self._check(self.lib.pfb_dirty(self.h, ctypes.byref(g), prec, nrow, nchan, _ptr(uvw), _ptr(freq),
                                       _ptr(band_of_chan), _ptr(vis), _ptr(wgt), _ptr(out), ws, self._stream()))
        return out, np.array(ws[:], dtype=np.float64)

    def pfb_psf(self, geom: Geometry, uvw, freq, band_of_chan, wgt=None, dtype=torch.float32, out=None):
        """I^psf on the 2nx x 2ny grid (centre (nx, ny)) and the per-band weight sums."""
        nrow, nchan = self._data(uvw, freq, band_of_chan)
        prec = _prec_real(wgt.dtype if wgt is not None else dtype)
        if wgt is not None:
            self._t(wgt, "wgt", _RDT[prec], (nrow, nchan))
        shape = (geom.nband, 2 * geom.nx, 2 * geom.ny)
        if out is None:
            out = torch.empty(shape, dtype=_RDT[prec], device=self.device)
        self._t(out, "psf_out", _RDT[prec], shape)
        ws = (ctypes.c_double * geom.nband)()
        g = geom.c()
        self._check(self.lib.pfb_psf(self.h, ctypes.byref(g), prec, nrow, nchan, _ptr(uvw), _ptr(freq),
                                     _ptr(band_of_chan), _ptr(wgt), _ptr(out), ws, self._stream()))
        return out, np.array(ws[:], dtype=np.float64)

    def pfb_hessian(self, geom: Geometry, uvw, freq, band_of_chan, x, wgt=None, out=None):
        """R^dagger Sigma^-1 R x (Eq. 3)."""
        nrow, nchan = self._data(uvw, freq, band_of_chan)
        prec = _prec_real(x.dtype)
        self._t(x, "x", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        if wgt is not None:
            self._t(wgt, "wgt", _RDT[prec], (nrow, nchan))
        if out is None:
            out = torch.empty_like(x)
        self._t(out, "y_out", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        g = geom.c()
        self._check(self.lib.pfb_hessian(self.h, ctypes.byref(g), prec, nrow, nchan, _ptr(uvw), _ptr(freq),
                                         _ptr(band_of_chan), _ptr(wgt), _ptr(x), _ptr(out), self._stream()))
        return out

    def pfb_hessian_host(self, geom: Geometry, uvw, freq, band_of_chan, x, wgt=None, out=None):
        """R^dagger Sigma^-1 R x (Eq. 3) from CPU tensors (pinned for asynchronous copies): the library
        copies the inputs in and each band of the result out while the later bands are computed.  out (a
        CPU tensor, pinned when allocated here) holds the result once the current CUDA stream is
        synchronised."""
        for name, t, dt in (("uvw", uvw, torch.float64), ("freq", freq, torch.float64),
                            ("band_of_chan", band_of_chan, torch.int32)):
            if t.dtype != dt or not t.is_contiguous() or t.device.type != "cpu":
                raise TypeError(f"{name} must be a contiguous {dt} CPU tensor")
        if uvw.ndim != 2 or uvw.shape[1] != 3:
            raise ValueError("uvw must be [nrow, 3]")
        nrow, nchan = uvw.shape[0], freq.shape[0]
        prec = _prec_real(x.dtype)
        shape = (geom.nband, geom.nx, geom.ny)
        for name, t, shp in (("x", x, shape), ("wgt", wgt, (nrow, nchan))):
            if t is not None and (t.dtype != _RDT[prec] or not t.is_contiguous() or t.device.type != "cpu"
                                  or tuple(t.shape) != tuple(shp)):
                raise TypeError(f"{name} must be a contiguous {_RDT[prec]} CPU tensor of shape {shp}")
        if out is None:
            out = torch.empty(shape, dtype=_RDT[prec], pin_memory=True)
        if out.dtype != _RDT[prec] or not out.is_contiguous() or out.device.type != "cpu" or \
                tuple(out.shape) != tuple(shape):
            raise TypeError(f"y_out must be a contiguous {_RDT[prec]} CPU tensor of shape {shape}")
        # the plan is keyed on these host pointers: hold the arrays so that their memory is not handed
        # to new arrays with other contents while the plan lives
        self._keep_host = (uvw, freq, band_of_chan)
        g = geom.c()
        self._check(self.lib.pfb_hessian_host(self.h, ctypes.byref(g), prec, nrow, nchan, _ptr(uvw), _ptr(freq),
                                              _ptr(band_of_chan), _ptr(wgt), _ptr(x), _ptr(out), self._stream()))
        return out

    def pfb_psf_conv(self, geom: Geometry, psf, x, out=None):
        """I^psf * x (Eq. 4), linear convolution."""
        prec = _prec_real(x.dtype)
        self._t(x, "x", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        self._t(psf, "psf", _RDT[prec], (geom.nband, 2 * geom.nx, 2 * geom.ny))
        if out is None:
            out = torch.empty_like(x)
        self._t(out, "y_out", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        g = geom.c()
        self._check(self.lib.pfb_psf_conv(self.h, ctypes.byref(g), prec, _ptr(psf), _ptr(x), _ptr(out),
                                          self._stream()))
        return out

    def pfb_step(self, geom: Geometry, params: StepParams, uvw, freq, band_of_chan, wgt, dirty, psf, wsum,
                 x, dual, stats: bool = True):
        """One preconditioned forward-backward step (Eqs. 6-7); x and dual are updated in place.
        Returns (n_hessian, stats) with stats = [objective, relative update, CG residual]."""
        nrow, nchan = self._data(uvw, freq, band_of_chan)
        prec = _prec_real(x.dtype)
        nb = bin(params.basis_mask).count("1")
        self._t(x, "x", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        self._t(dirty, "dirty", _RDT[prec], (geom.nband, geom.nx, geom.ny))
        self._t(psf, "psf", _RDT[prec], (geom.nband, 2 * geom.nx, 2 * geom.ny))
        self._t(dual, "dual", _RDT[prec], (nb, geom.nband, geom.nx, geom.ny))
        if wgt is not None:
            self._t(wgt, "wgt", _RDT[prec], (nrow, nchan))
        ws = (ctypes.c_double * geom.nband)(*[float(v) for v in wsum])
        nh = ctypes.c_int64(0)
        st = (ctypes.c_double * 3)()
        g, p = geom.c(), params.c()
        self._check(self.lib.pfb_step(self.h, ctypes.byref(g), prec, ctypes.byref(p), nrow, nchan, _ptr(uvw),
                                      _ptr(freq), _ptr(band_of_chan), _ptr(wgt), _ptr(dirty), _ptr(psf), ws,
                                      _ptr(x), _ptr(dual), ctypes.byref(nh), st if stats else None,
                                      self._stream()))
        return int(nh.value), np.array(st[:]) if stats else None

    def pfb_clean(self, geom: Geometry, params: StepParams, uvw, freq, band_of_chan, vis, wgt=None,
                  max_outer: int = 20, tol: float = 0.0, x=None, dual=None):
        """A whole solve: I^psf (2x field), I^d, then up to max_outer steps until the relative
        update is <= tol.  x and dual (zeros if None) are updated in place.  Returns a dict with
        x, dual, dirty, psf, wsum, n_outer, n_hessian and history ([n_outer][3] step stats)."""
        nrow, nchan = self._data(uvw, freq, band_of_chan)
        prec = _prec_cx(vis.dtype)
        rdt = _RDT[prec]
        self._t(vis, "vis", _CDT[prec], (nrow, nchan))
        if wgt is not None:
            self._t(wgt, "wgt", rdt, (nrow, nchan))
        img = (geom.nband, geom.nx, geom.ny)
        nb = bin(params.basis_mask).count("1")
        if x is None:
            x = torch.zeros(img, dtype=rdt, device=self.device)
        if dual is None:
            dual = torch.zeros((nb,) + img, dtype=rdt, device=self.device)
        self._t(x, "x", rdt, img)
        self._t(dual, "dual", rdt, (nb,) + img)
        dirty = torch.empty(img, dtype=rdt, device=self.device)
        psf = torch.empty((geom.nband, 2 * geom.nx, 2 * geom.ny), dtype=rdt, device=self.device)
        ws = (ctypes.c_double * geom.nband)()
        hist = (ctypes.c_double * (3 * max(max_outer, 1)))()
        no, nh = ctypes.c_int32(0), ctypes.c_int64(0)
        g, p = geom.c(), params.c()
        self._check(self.lib.pfb_clean(self.h, ctypes.byref(g), prec, ctypes.byref(p), int(max_outer), float(tol),
                                       nrow, nchan, _ptr(uvw), _ptr(freq), _ptr(band_of_chan), _ptr(vis),
                                       _ptr(wgt), _ptr(dirty), _ptr(psf), ws, _ptr(x), _ptr(dual),
                                       ctypes.byref(no), ctypes.byref(nh), hist, self._stream()))
        k = int(no.value)
        return {"x": x, "dual": dual, "dirty": dirty, "psf": psf, "wsum": np.array(ws[:], dtype=np.float64),
                "n_outer": k, "n_hessian": int(nh.value),
                "history": np.array(hist[:3 * k], dtype=np.float64).reshape(k, 3)}

    def pfb_step_bound(self, geom: Geometry, params: StepParams, uvw, freq, band_of_chan, wgt, psf, wsum,
                       iters: int = 8, z0=None) -> float:
        """lambda_max(U^-1 H) by `iters` power iterations (the step converges for gamma < 2 / it)."""
        nrow, nchan = self._data(uvw, freq, band_of_chan)
        prec = _prec_real(psf.dtype)
        rdt = _RDT[prec]
        if wgt is not None:
            self._t(wgt, "wgt", rdt, (nrow, nchan))
        self._t(psf, "psf", rdt, (geom.nband, 2 * geom.nx, 2 * geom.ny))
        if z0 is not None:
            self._t(z0, "z0", rdt, (geom.nband, geom.nx, geom.ny))
        ws = (ctypes.c_double * geom.nband)(*[float(v) for v in wsum])
        out = ctypes.c_double(0)
        g, p = geom.c(), params.c()
        self._check(self.lib.pfb_step_bound(self.h, ctypes.byref(g), prec, ctypes.byref(p), nrow, nchan, _ptr(uvw),
                                            _ptr(freq), _ptr(band_of_chan), _ptr(wgt), _ptr(psf), ws, _ptr(z0),
                                            int(iters), ctypes.byref(out), self._stream()))
        return float(out.value)

    def pfb_last_step_bound(self) -> tuple[float, float]:
        """(lambda_max, gamma) of the last step-bound estimate / safe-gamma solve of this context."""
        lm, ga = ctypes.c_double(0), ctypes.c_double(0)
        self._check(self.lib.pfb_last_step_bound(self.h, ctypes.byref(lm), ctypes.byref(ga)))
        return float(lm.value), float(ga.value)

    def pfb_plan_reset(self):
        """Drop cached plans (after changing uvw/freq/band_of_chan in place)."""
        self._check(self.lib.pfb_plan_reset(self.h))
        self._keep.clear()


_default: dict[int, Context] = {}
_lock = threading.Lock()


def default_context(device: int | None = None) -> Context:
    d = torch.cuda.current_device() if device is None else device
    with _lock:
        if d not in _default:
            _default[d] = Context(d)
        return _default[d]


def version() -> str:
    return _lib.load().pfb_version().decode()
