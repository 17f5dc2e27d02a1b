"""Seeded synthetic inputs for the measurement-operator workloads.

This module draws random numbers and builds array geometry only: antenna
layouts, uvw tracks from Earth-rotation synthesis, channel frequencies, the
channel-to-band map, pixel sizes, sky models on the pixel grid, noise and
weights. It holds none of the imaging arithmetic (no measurement equation, no
gridding, no FFT): the visibilities of a sky model are formed by whichever
operator the caller is testing, and the noise drawn here is added on top.

Both the FP64 oracle and the CUDA path are fed from these generators, and
nothing else is shared between them.

Geometry conventions (Thompson, Moran & Swenson, "Interferometry and Synthesis
in Radio Astronomy", ch. 4):
  * local ENU -> equatorial XYZ at site latitude phi:
        X = -sin(phi) N + cos(phi) U,  Y = E,  Z = cos(phi) N + sin(phi) U
  * XYZ baseline -> (u, v, w) at hour angle H and declination delta:
        u =  sin H X + cos H Y
        v = -sin d cos H X + sin d sin H Y + cos d Z
        w =  cos d cos H X - cos d sin H Y + sin d Z
Rows are stored time-major (all baselines of one integration, then the next),
the usual Measurement Set order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299_792_458.0
ARCSEC = math.pi / (180.0 * 3600.0)


@dataclasses.dataclass
class Observation:
    """One synthetic observation: everything the operators take except the image."""
    uvw: np.ndarray            # [nrow, 3] float64 metres
    freq: np.ndarray           # [nchan] float64 Hz
    band_of_chan: np.ndarray   # [nchan] int32
    nx: int
    ny: int
    dl: float                  # pixel size in l (radians)
    dm: float                  # pixel size in m (radians)
    nband: int

    @property
    def nrow(self) -> int:
        return int(self.uvw.shape[0])

    @property
    def nchan(self) -> int:
        return int(self.freq.shape[0])

    @property
    def nvis(self) -> int:
        return self.nrow * self.nchan


def enu_to_xyz(enu: np.ndarray, lat: float) -> np.ndarray:
    e, n, u = enu[:, 0], enu[:, 1], enu[:, 2]
    x = -math.sin(lat) * n + math.cos(lat) * u
    y = e
    z = math.cos(lat) * n + math.sin(lat) * u
    return np.stack([x, y, z], axis=1)


def baseline_pairs(n_ant: int) -> tuple[np.ndarray, np.ndarray]:
    a1, a2 = np.triu_indices(n_ant, k=1)
    return a1.astype(np.int64), a2.astype(np.int64)


def uvw_tracks(xyz: np.ndarray, hour_angles: np.ndarray, dec: float) -> np.ndarray:
    """uvw [ntime*nbl, 3] (metres) for all baselines at each hour angle, time-major."""
    a1, a2 = baseline_pairs(xyz.shape[0])
    b = xyz[a2] - xyz[a1]                      # [nbl, 3]
    bx, by, bz = b[:, 0][None, :], b[:, 1][None, :], b[:, 2][None, :]
    h = hour_angles[:, None]
    sh, ch = np.sin(h), np.cos(h)
    sd, cd = math.sin(dec), math.cos(dec)
    u = sh * bx + ch * by
    v = -sd * ch * bx + sd * sh * by + cd * bz
    w = cd * ch * bx - cd * sh * by + sd * bz
    return np.stack([u, v, w], axis=-1).reshape(-1, 3).astype(np.float64)


def contiguous_bands(nchan: int, nband: int) -> np.ndarray:
    """Equal contiguous channel groups: band b = floor(chan * nband / nchan)."""
    return (np.arange(nchan, dtype=np.int64) * nband // nchan).astype(np.int32)


def max_uv_lambda(uvw: np.ndarray, freq: np.ndarray) -> float:
    """Largest |(u, v)| in wavelengths over all rows and channels (geometry only)."""
    r = np.sqrt(uvw[:, 0] ** 2 + uvw[:, 1] ** 2).max()
    return float(r * freq.max() / C_LIGHT)


# ---------------------------------------------------------------- config 1
def tiny_observation(seed: int = 1, nx: int = 64, ny: int = 64, n_ant: int = 16,
                     ntime: int = 17, nchan: int = 4, nband: int = 1,
                     f_lo: float = 1.0e9, f_hi: float = 1.1e9,
                     disk_diameter_m: float = 1000.0, dec_deg: float = -30.0,
                     lat_deg: float = -30.7, ha_span_h: float = 8.0) -> Observation:
    """Tiny FP64 case: 16 antennas uniform in a 1 km disk, 17 hour angles over
    -4 h..+4 h, 4 channels over 1.0-1.1 GHz, pixel size at Nyquist for the
    longest baseline at the top frequency (dl = 1 / (2 u_max))."""
    rng = np.random.default_rng(seed)
    r = 0.5 * disk_diameter_m * np.sqrt(rng.uniform(0.0, 1.0, n_ant))
    th = rng.uniform(0.0, 2.0 * math.pi, n_ant)
    enu = np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n_ant)], axis=1)
    xyz = enu_to_xyz(enu, math.radians(lat_deg))
    ha = np.linspace(-0.5 * ha_span_h, 0.5 * ha_span_h, ntime) * (math.pi / 12.0)
    uvw = uvw_tracks(xyz, ha, math.radians(dec_deg))
    freq = np.linspace(f_lo, f_hi, nchan).astype(np.float64)
    umax = max_uv_lambda(uvw, freq)
    dl = 1.0 / (2.0 * umax)
    return Observation(uvw=uvw, freq=freq, band_of_chan=contiguous_bands(nchan, nband),
                       nx=nx, ny=ny, dl=dl, dm=dl, nband=nband)


# ---------------------------------------------------------------- config 2 family
def meerkat_like_layout(rng: np.random.Generator, n_core: int = 48, n_outer: int = 16,
                        core_radius_m: float = 1000.0, outer_radius_m: float = 4000.0) -> np.ndarray:
    """Synthetic (not any real array's) layout: a Gaussian core truncated at
    core_radius_m plus antennas spread uniformly in radius out to outer_radius_m."""
    pts = []
    while len(pts) < n_core:
        p = rng.normal(0.0, 0.45 * core_radius_m, 2)
        if np.hypot(p[0], p[1]) <= core_radius_m:
            pts.append(p)
    core = np.array(pts)
    r = rng.uniform(core_radius_m, outer_radius_m, n_outer)
    th = rng.uniform(0.0, 2.0 * math.pi, n_outer)
    outer = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    en = np.concatenate([core, outer], axis=0)
    return np.concatenate([en, np.zeros((en.shape[0], 1))], axis=1)


def meerkat_like_observation(seed: int = 2, ntime: int = 450, dt_s: float = 8.0,
                             nchan: int = 256, nband: int = 4,
                             f_lo: float = 0.856e9, f_hi: float = 1.712e9,
                             nx: int = 4096, ny: int = 4096, cell_arcsec: float = 1.5,
                             dec_deg: float = -30.0, lat_deg: float = -30.7,
                             n_core: int = 48, n_outer: int = 16) -> Observation:
    """MeerKAT-like wide-field continuum geometry: 64 antennas (2016 baselines)
    x 450 integrations of 8 s centred on transit, 256 channels over
    0.856-1.712 GHz in 4 contiguous bands, 4096^2 pixels of 1.5 arcsec."""
    rng = np.random.default_rng(seed)
    enu = meerkat_like_layout(rng, n_core, n_outer)
    xyz = enu_to_xyz(enu, math.radians(lat_deg))
    t = (np.arange(ntime) - 0.5 * (ntime - 1)) * dt_s
    ha = t * (2.0 * math.pi / 86164.0905)
    uvw = uvw_tracks(xyz, ha, math.radians(dec_deg))
    # channel centres of nchan equal channels spanning [f_lo, f_hi]
    df = (f_hi - f_lo) / nchan
    freq = (f_lo + (np.arange(nchan) + 0.5) * df).astype(np.float64)
    d = cell_arcsec * ARCSEC
    return Observation(uvw=uvw, freq=freq, band_of_chan=contiguous_bands(nchan, nband),
                       nx=nx, ny=ny, dl=d, dm=d, nband=nband)


def subset_rows(obs: Observation, rows: np.ndarray) -> Observation:
    return dataclasses.replace(obs, uvw=np.ascontiguousarray(obs.uvw[rows]))


# ---------------------------------------------------------------- sky models
def point_source_image(rng: np.random.Generator, nband: int, nx: int, ny: int, nsrc: int,
                       flux: str = "uniform", fmin: float = 0.1, fmax: float = 1.0,
                       pareto_index: float = 1.5, spectral: bool = False,
                       band_freqs: np.ndarray | None = None) -> np.ndarray:
    """Point sources at distinct uniform-random pixels, image [nband][nx][ny] float64.

    flux='uniform': U(fmin, fmax).  flux='pareto': a power law N(>S) ~ S^-index
    truncated to [fmin, fmax] (inverse-CDF draw).  With spectral=True each source
    gets a spectral index ~ N(-0.7, 0.2) about the first band's frequency."""
    npix = nx * ny
    idx = rng.choice(npix, size=nsrc, replace=False)
    if flux == "uniform":
        s = rng.uniform(fmin, fmax, nsrc)
    elif flux == "pareto":
        a = pareto_index
        uu = rng.uniform(0.0, 1.0, nsrc)
        lo, hi = fmin ** (-a), fmax ** (-a)
        s = (lo - uu * (lo - hi)) ** (-1.0 / a)
    else:
        raise ValueError(flux)
    img = np.zeros((nband, npix), dtype=np.float64)
    if spectral and band_freqs is not None and nband > 1:
        alpha = rng.normal(-0.7, 0.2, nsrc)
        for b in range(nband):
            img[b, idx] = s * (band_freqs[b] / band_freqs[0]) ** alpha
    else:
        img[:, idx] = s[None, :]
    return img.reshape(nband, nx, ny)


def gaussian_blob_image(rng: np.random.Generator, nband: int, nx: int, ny: int, nblob: int,
                        fwhm_px: tuple[float, float] = (5.0, 60.0), fmin: float = 0.01,
                        fmax: float = 0.1) -> np.ndarray:
    """Extended circular Gaussian sources sampled on the pixel grid (peak flux
    ~U(fmin, fmax), FWHM ~U(fwhm_px)), image [nband][nx][ny] float64."""
    img = np.zeros((nx, ny), dtype=np.float64)
    ii = np.arange(nx)[:, None]
    jj = np.arange(ny)[None, :]
    for _ in range(nblob):
        ci, cj = rng.uniform(0, nx), rng.uniform(0, ny)
        fw = rng.uniform(*fwhm_px)
        s = fw / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        pk = rng.uniform(fmin, fmax)
        r = int(4 * s) + 1
        i0, i1 = max(0, int(ci) - r), min(nx, int(ci) + r + 1)
        j0, j1 = max(0, int(cj) - r), min(ny, int(cj) + r + 1)
        img[i0:i1, j0:j1] += pk * np.exp(-((ii[i0:i1] - ci) ** 2 + (jj[:, j0:j1] - cj) ** 2) / (2 * s * s))
    return np.repeat(img[None], nband, axis=0)


def sparse_random_image(rng: np.random.Generator, nband: int, nx: int, ny: int,
                        density: float = 0.01) -> np.ndarray:
    """Non-negative image with a fraction `density` of pixels ~U(0,1), rest 0."""
    m = rng.uniform(0.0, 1.0, (nband, nx, ny)) < density
    return np.where(m, rng.uniform(0.0, 1.0, (nband, nx, ny)), 0.0)


# ---------------------------------------------------------------- data-side draws
def complex_noise(rng: np.random.Generator, shape, variance: float = 0.01) -> np.ndarray:
    """Complex Gaussian noise with total variance `variance` per visibility,
    split equally between the real and imaginary parts."""
    s = math.sqrt(0.5 * variance)
    return rng.normal(0.0, s, shape) + 1j * rng.normal(0.0, s, shape)


def weighted_noise(rng: np.random.Generator, wgt: np.ndarray) -> np.ndarray:
    """Complex noise with per-component standard deviation 1/sqrt(W)."""
    s = 1.0 / np.sqrt(wgt)
    return rng.normal(0.0, 1.0, wgt.shape) * s + 1j * rng.normal(0.0, 1.0, wgt.shape) * s


def uniform_weights(rng: np.random.Generator, shape, lo: float = 0.5, hi: float = 1.5,
                    dtype=np.float64) -> np.ndarray:
    return rng.uniform(lo, hi, shape).astype(dtype)


def random_vis(rng: np.random.Generator, shape) -> np.ndarray:
    """Unit-variance complex Gaussian visibilities (adjoint-test vectors)."""
    return (rng.normal(0.0, 1.0, shape) + 1j * rng.normal(0.0, 1.0, shape)) / math.sqrt(2.0)


def band_centre_freqs(freq: np.ndarray, band_of_chan: np.ndarray, nband: int) -> np.ndarray:
    return np.array([freq[band_of_chan == b].mean() for b in range(nband)])


def poisson_arrivals(rng: np.random.Generator, n: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))


def log_uniform_int(rng: np.random.Generator, lo: float, hi: float, size=None) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size)).astype(np.int64)
