"""Shared helpers of the GPU tests: device copies of synthetic inputs and error norms."""
import numpy as np
import torch

from paper_2101_08072_gb300 import synth

# Tolerances on the relative L2 error against the FP64 oracle.  The FP32 path must
# reach 3e-5 when asked for epsilon = 1e-5; the FP64 path 1e-9 at epsilon = 1e-10.
EPS32, TOL32 = 1e-5, 3e-5
EPS64, TOL64 = 1e-10, 1e-9


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def dev_obs(obs: synth.Observation, device="cuda"):
    return (torch.from_numpy(np.ascontiguousarray(obs.uvw)).to(device),
            torch.from_numpy(np.ascontiguousarray(obs.freq)).to(device),
            torch.from_numpy(np.ascontiguousarray(obs.band_of_chan, dtype=np.int32)).to(device))


def geometry(obs: synth.Observation, eps: float, flags: int = 0):
    from paper_2101_08072_gb300 import Geometry
    return Geometry(nx=obs.nx, ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=eps, flags=flags)


def real_t(a, prec, device="cuda"):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64 if prec == 64 else np.float32)).to(device)


def cx_t(a, prec, device="cuda"):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128 if prec == 64 else np.complex64)).to(device)


def wide_observation(seed=31, nx=96, ny=160, nband=3, band_of_chan=(0, 0, 0, 1, 2, 2, 2, 2),
                     uv_scale=6.0):
    """A non-square, multi-tile image with uneven bands and a strong w term: the
    tiny array's baselines are stretched so that w (n - 1) reaches several turns."""
    nchan = len(band_of_chan)
    obs = synth.tiny_observation(seed=seed, nx=nx, ny=ny, nchan=nchan, nband=nband)
    uvw = obs.uvw * uv_scale
    umax = synth.max_uv_lambda(uvw, obs.freq)
    dl = 1.0 / (2.2 * umax)
    return synth.Observation(uvw=uvw, freq=obs.freq, band_of_chan=np.array(band_of_chan, dtype=np.int32),
                             nx=nx, ny=ny, dl=dl, dm=dl * 1.1, nband=nband)
