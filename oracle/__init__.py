"""FP64 oracle for the pfb-clean hot path (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  The product path (paper_2101_08072_gb300) never
imports, links or runs it, and this package imports nothing from the product.

What it computes, each from the paper's definitions (Bester et al. 2021,
"A practical preconditioner for wide-field continuum imaging of radio
interferometric data"):

  degrid      R x  (Eq. 1, Section 2): direct DFT with the exact n-1 term and 1/n
  grid        R^dagger Sigma^-1 y (Eq. 3): the real adjoint of R, weighted
  dirty       I^d = R^dagger Sigma^-1 V (Eq. 3)
  psf         I^psf = R'^dagger Sigma^-1 1 on a 2nx x 2ny grid (Eq. 4, Eq. 8)
  hessian     R^dagger Sigma^-1 R x (Eq. 3)
  psf_conv    I^psf * x as a linear convolution (Eq. 4): direct sum or padded FFT
  cg          conjugate gradient for U delta = IR, U = I^psf* + sigma Id (Eq. 6, Eq. 8)
  prox        Condat-Vu primal-dual for Eq. 7 with r(x) of Eq. 9
  step        one preconditioned forward-backward step (Eqs. 6-7); optionally with
              the approximate gradient of Eq. 4 (I^psf * x in place of H x)
  step_bound  lambda_max(U^-1 H) by power iteration (the step size bound of Eqs. 6-7)
  clean       a whole solve: PSF, dirty image, then steps until the relative update
              reaches a tolerance (optionally with gamma capped at 1.9 / lambda_max)
  daubechies  db1..db6 filters by spectral factorisation, periodised DWT (Eq. 9's Psi)

Parity status: R, R^dagger, I^d, I^psf, the Hessian, the PSF convolution, CG,
the prox, the wavelets and the gradient are pinned by tests/test_oracle_pins.py
(closed forms, library-routine special cases, invariants, brute force).  The
composed step is pinned at lam = 0 with CG run to convergence, where the prox is
the identity, against a dense computation of x + gamma U^-1 (I^d - H x) / wbar;
so are the fixed point at the true image, the reduction of the approximate
gradient to the exact one at w = 0 and the stopping rule; CG at a fixed
iteration count k is pinned as the U-norm minimiser over the k-dimensional
Krylov space.  With lam > 0 the primal-dual iterates at a fixed, unconverged
count, and so the step and clean iterates, have no printed value in the paper
and no closed form: those iterates are "parity unpinned" (their parts are pinned).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NO_DIVIDE_BY_N = 1
NO_WTERM = 2


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc + OpenMP (plain C, FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64, u32 = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint
        lib.oracle_degrid.argtypes = [i32, i32, f64, f64, f64, f64, i32, i64, i32, P, P, P, P, u32, i64, P, P]
        lib.oracle_grid.argtypes = [i32, i32, f64, f64, f64, f64, i32, i64, i32, P, P, P, P, P, u32, i64, P, P]
        lib.oracle_wsum.argtypes = [i32, i64, i32, P, P, P]
        lib.oracle_psf_conv_direct.argtypes = [i32, i32, i32, P, P, P]
        lib.oracle_num_threads.restype = i32
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------ R and R^dagger
def degrid(uvw, freq, band_of_chan, image, dl, dm, flags=0, rows=None, l0=0.0, m0=0.0):
    """R x (Eq. 1).  image [nband][nx][ny] -> vis [nrow][nchan] complex128.
    rows: optional row indices; then only those rows are returned, [len(rows)][nchan].
    (l0, m0): direction cosines of the image centre (a facet away from the phase centre)."""
    lib = _load()
    uvw, freq = _c(uvw, np.float64), _c(freq, np.float64)
    boc, image = _c(band_of_chan, np.int32), _c(image, np.float64)
    nband, nx, ny = image.shape
    nrow, nchan = uvw.shape[0], freq.shape[0]
    sel = None if rows is None else _c(rows, np.int64)
    nout = nrow if sel is None else sel.shape[0]
    out = np.zeros((nout, nchan, 2), dtype=np.float64)
    lib.oracle_degrid(nx, ny, dl, dm, l0, m0, nband, nrow, nchan, _p(uvw), _p(freq), _p(boc), _p(image),
                      flags, 0 if sel is None else sel.shape[0], _p(sel), _p(out))
    return out[..., 0] + 1j * out[..., 1]


def grid(uvw, freq, band_of_chan, vis, wgt, nx, ny, dl, dm, nband, flags=0, pix=None, l0=0.0, m0=0.0):
    """R^dagger Sigma^-1 y (Eq. 3).  vis [nrow][nchan] complex, wgt same shape or None.
    pix: optional flat indices b*nx*ny + i*ny + j; then returns [len(pix)].
    (l0, m0): direction cosines of the image centre (a facet away from the phase centre)."""
    lib = _load()
    uvw, freq = _c(uvw, np.float64), _c(freq, np.float64)
    boc = _c(band_of_chan, np.int32)
    v = np.ascontiguousarray(np.stack([np.real(vis), np.imag(vis)], axis=-1), dtype=np.float64)
    w = None if wgt is None else _c(wgt, np.float64)
    nrow, nchan = uvw.shape[0], freq.shape[0]
    sel = None if pix is None else _c(pix, np.int64)
    out = np.zeros(nband * nx * ny if sel is None else sel.shape[0], dtype=np.float64)
    lib.oracle_grid(nx, ny, dl, dm, l0, m0, nband, nrow, nchan, _p(uvw), _p(freq), _p(boc), _p(v), _p(w),
                    flags, 0 if sel is None else sel.shape[0], _p(sel), _p(out))
    return out.reshape(nband, nx, ny) if sel is None else out


def wsum(band_of_chan, wgt, nrow, nband):
    lib = _load()
    boc = _c(band_of_chan, np.int32)
    w = None if wgt is None else _c(wgt, np.float64)
    out = np.zeros(nband, dtype=np.float64)
    lib.oracle_wsum(nband, nrow, boc.shape[0], _p(boc), _p(w), _p(out))
    return out


def dirty(uvw, freq, band_of_chan, vis, wgt, nx, ny, dl, dm, nband, flags=0, l0=0.0, m0=0.0):
    """I^d = R^dagger Sigma^-1 V (Eq. 3) and the per-band weight sums."""
    img = grid(uvw, freq, band_of_chan, vis, wgt, nx, ny, dl, dm, nband, flags, l0=l0, m0=m0)
    return img, wsum(band_of_chan, wgt, uvw.shape[0], nband)


def psf(uvw, freq, band_of_chan, wgt, nx, ny, dl, dm, nband, flags=0, l0=0.0, m0=0.0):
    """I^psf: the adjoint applied to Sigma^-1 1 on a 2nx x 2ny grid with the same
    pixel size, centre pixel (nx, ny) at (l0, m0).  Unnormalised: at the phase
    centre its peak is the per-band weight sum."""
    ones = np.ones((uvw.shape[0], freq.shape[0]), dtype=np.complex128)
    img = grid(uvw, freq, band_of_chan, ones, wgt, 2 * nx, 2 * ny, dl, dm, nband, flags, l0=l0, m0=m0)
    return img, wsum(band_of_chan, wgt, uvw.shape[0], nband)


def hessian(uvw, freq, band_of_chan, wgt, x, dl, dm, flags=0, l0=0.0, m0=0.0):
    """R^dagger Sigma^-1 R x (Eq. 3)."""
    nband, nx, ny = x.shape
    rx = degrid(uvw, freq, band_of_chan, x, dl, dm, flags, l0=l0, m0=m0)
    return grid(uvw, freq, band_of_chan, rx, wgt, nx, ny, dl, dm, nband, flags, l0=l0, m0=m0)


# ------------------------------------------------------------------ PSF convolution
def psf_conv_direct(psf_img, x):
    """(I^psf * x)[b,i,j] = sum psf[b, i-i'+nx, j-j'+ny] x[b,i',j'] (Eq. 4), direct sum."""
    lib = _load()
    p, xx = _c(psf_img, np.float64), _c(x, np.float64)
    nband, nx, ny = xx.shape
    y = np.zeros_like(xx)
    lib.oracle_psf_conv_direct(nx, ny, nband, _p(p), _p(xx), _p(y))
    return y


def psf_spectrum(psf_img):
    """FFT of the PSF with its centre moved to index (0, 0): the transfer function
    of the linear convolution on the 2nx x 2ny zero-padded grid."""
    return np.fft.fft2(np.fft.ifftshift(np.asarray(psf_img, dtype=np.float64), axes=(1, 2)))


def psf_conv(psf_img, x, spectrum=None):
    """Eq. 4's I^psf * x by zero padding to 2nx x 2ny and the FFT convolution
    theorem; exact (to rounding) for the linear convolution defined above."""
    x = np.asarray(x, dtype=np.float64)
    nband, nx, ny = x.shape
    P = psf_spectrum(psf_img) if spectrum is None else spectrum
    xp = np.zeros((nband, 2 * nx, 2 * ny))
    xp[:, :nx, :ny] = x
    return np.real(np.fft.ifft2(np.fft.fft2(xp) * P))[:, :nx, :ny]


# ------------------------------------------------------------------ preconditioner U
def u_apply(spec_sym, sigma, x):
    """U x = I^psf_sym * x + sigma x (Eq. 8).  spec_sym is the real part of the PSF
    spectrum: the convolution with the PSF symmetrised about its centre, which is
    the symmetric part of I^psf* (equal to it when w = 0)."""
    return psf_conv(None, x, spectrum=spec_sym) + sigma * x


def cg(spec_sym, sigma, b, iters, tol=0.0):
    """Hestenes-Stiefel conjugate gradient for U delta = b (Eq. 6 needs U^-1 grad f),
    run per band from delta_0 = 0.  Returns (delta, relative residual norm per band)."""
    b = np.asarray(b, dtype=np.float64)
    nband = b.shape[0]
    out = np.zeros_like(b)
    res = np.zeros(nband)
    for k in range(nband):
        bk = b[k:k + 1]
        x = np.zeros_like(bk)
        r = bk.copy()
        p = r.copy()
        rr = float(np.vdot(r, r))
        bnorm = math.sqrt(rr)
        for _ in range(iters):
            if rr == 0.0 or math.sqrt(rr) <= tol * bnorm:
                break
            ap = u_apply(spec_sym[k:k + 1], sigma, p)
            alpha = rr / float(np.vdot(p, ap))
            x = x + alpha * p
            r = r - alpha * ap
            rr_new = float(np.vdot(r, r))
            p = r + (rr_new / rr) * p
            rr = rr_new
        out[k] = x[0]
        res[k] = math.sqrt(rr) / bnorm if bnorm > 0 else 0.0
    return out, res


# ------------------------------------------------------------------ Daubechies dictionary
def daubechies(N: int) -> np.ndarray:
    """Low-pass filter of the Daubechies wavelet with N vanishing moments (length 2N),
    by spectral factorisation (Daubechies 1988):
        |m0|^2 = cos^{2N}(w/2) P(sin^2(w/2)),  P(y) = sum_{k<N} C(N-1+k, k) y^k.
    Each root y_k of P gives z^2 - (2 - 4 y_k) z + 1 = 0; the root inside the unit
    circle is kept (minimum phase).  h = coefficients, highest power of z first, of
    (z + 1)^N prod(z - z_k), scaled so that sum h = sqrt(2)."""
    if N == 1:
        return np.array([1.0, 1.0]) / math.sqrt(2.0)
    coeffs = [math.comb(N - 1 + k, k) for k in range(N)]
    yroots = np.roots(coeffs[::-1])
    zroots = []
    for y in yroots:
        a = 1.0 - 2.0 * y
        s = np.sqrt(a * a - 1.0 + 0j)
        z1, z2 = a + s, a - s
        zroots.append(z1 if abs(z1) < 1.0 else z2)
    h = np.real(np.poly(np.concatenate([-np.ones(N), np.array(zroots)])))
    return h * (math.sqrt(2.0) / h.sum())


def highpass(h: np.ndarray) -> np.ndarray:
    """Quadrature-mirror high-pass: g_k = (-1)^k h_{L-1-k}."""
    L = h.shape[0]
    return np.array([(-1) ** k * h[L - 1 - k] for k in range(L)])


def _dwt1(x, h, g, axis):
    """One level of the periodised orthonormal DWT along `axis`:
    a[k] = sum_n h[n] x[(2k+n) mod N], d[k] = sum_n g[n] x[(2k+n) mod N]."""
    x = np.moveaxis(x, axis, 0)
    N = x.shape[0]
    a = np.zeros((N // 2,) + x.shape[1:])
    d = np.zeros_like(a)
    for k in range(N // 2):
        for n in range(h.shape[0]):
            a[k] += h[n] * x[(2 * k + n) % N]
            d[k] += g[n] * x[(2 * k + n) % N]
    return np.moveaxis(np.concatenate([a, d], axis=0), 0, axis)


def _idwt1(c, h, g, axis):
    """Transpose (= inverse, the transform being orthonormal) of _dwt1."""
    c = np.moveaxis(c, axis, 0)
    N = c.shape[0]
    a, d = c[:N // 2], c[N // 2:]
    x = np.zeros_like(c)
    for k in range(N // 2):
        for n in range(h.shape[0]):
            x[(2 * k + n) % N] += h[n] * a[k] + g[n] * d[k]
    return np.moveaxis(x, 0, axis)


def dwt2(img, h, nlevel):
    """Multi-level 2-D periodised DWT of one [nx][ny] image, Mallat layout: at each
    level the current low-pass block [0:n, 0:m] is transformed along axis 0 then
    axis 1 and the recursion continues on [0:n/2, 0:m/2]."""
    c = np.array(img, dtype=np.float64)
    g = highpass(h)
    n, m = c.shape
    for _ in range(nlevel):
        blk = _dwt1(c[:n, :m], h, g, 0)
        c[:n, :m] = _dwt1(blk, h, g, 1)
        n, m = n // 2, m // 2
    return c


def idwt2(coef, h, nlevel):
    c = np.array(coef, dtype=np.float64)
    g = highpass(h)
    n, m = c.shape[0] >> (nlevel - 1), c.shape[1] >> (nlevel - 1)
    for _ in range(nlevel):
        blk = _idwt1(c[:n, :m], h, g, 1)
        c[:n, :m] = _idwt1(blk, h, g, 0)
        n, m = 2 * n, 2 * m
    return c


def basis_list(basis_mask: int):
    """Bit 0 = Dirac, bit k (1..6) = Daubechies db_k (Eq. 9's dictionary)."""
    return [k for k in range(7) if basis_mask >> k & 1]


def psi_adjoint(x, bases, nlevel):
    """Psi^dagger x: analysis coefficients [nbasis][nband][nx][ny] of the dictionary
    Psi = [Psi_1 ... Psi_K] / sqrt(K) (each Psi_k orthonormal, so ||Psi|| = 1)."""
    K = len(bases)
    out = np.zeros((K,) + x.shape)
    for t, k in enumerate(bases):
        for b in range(x.shape[0]):
            out[t, b] = x[b] if k == 0 else dwt2(x[b], daubechies(k), nlevel)
    return out / math.sqrt(K)


def psi(v, bases, nlevel):
    """Psi v = sum_k Psi_k v_k / sqrt(K) (synthesis)."""
    K = len(bases)
    out = np.zeros(v.shape[1:])
    for t, k in enumerate(bases):
        for b in range(v.shape[1]):
            out[b] += v[t, b] if k == 0 else idwt2(v[t, b], daubechies(k), nlevel)
    return out / math.sqrt(K)


def l21(coef):
    """||c||_{2,1}: l2 over imaging bands for each (basis, coefficient), l1 over the rest."""
    return float(np.sqrt((coef ** 2).sum(axis=1)).sum())


# ------------------------------------------------------------------ prox (Eq. 7)
@dataclass
class Params:
    gamma: float = 1.0
    sigma: float = 1e-3
    lam: float = 1e-4
    cg_iters: int = 50
    cg_tol: float = 0.0
    pd_iters: int = 100
    nlevel: int = 3
    basis_mask: int = 1
    unorm: float = 0.0          # ||U||; <= 0 means max|Re spectrum| + sigma
    approx_gradient: bool = False   # Eq. 4: I^psf * x stands in for H x
    safe_gamma: bool = False    # clean: cap gamma at SAFE_GAMMA_FACTOR / lambda_max(U^-1 H)


def unorm_of(spec_sym, sigma):
    return float(np.abs(spec_sym).max()) + sigma


def prox(xbar, v, spec_sym, p: Params):
    """Condat-Vu primal-dual iterations (Condat 2013) for Eq. 7 with r of Eq. 9:
        argmin_x  lam ||Psi^dagger x||_{2,1} + iota_+(x) + (1/2 gamma)(x - xbar)^T U (x - xbar).
    Smooth part F(x) = (1/2 gamma)(x-xbar)^T U (x-xbar), grad F = U(x-xbar)/gamma,
    Lipschitz L = ||U||/gamma; dual step 1, primal step tau = 0.98/(L/2 + 1), so
    1/tau - ||Psi||^2 >= L/2 with ||Psi|| = 1.  Each iteration:
        x~ = max(0, x - tau (grad F(x) + Psi v))
        v~ = v + Psi^dagger (2 x~ - x)
        v  = v~_g min(1, lam / ||v~_g||_2) per group g  (prox of the conjugate of lam||.||_{2,1})
        x  = x~
    Starts from x = max(xbar, 0) and the dual passed in."""
    bases = basis_list(p.basis_mask)
    unorm = p.unorm if p.unorm > 0 else unorm_of(spec_sym, p.sigma)
    L = unorm / p.gamma
    tau = 0.98 / (0.5 * L + 1.0)
    x = np.maximum(xbar, 0.0)
    v = np.array(v, dtype=np.float64)
    for _ in range(p.pd_iters):
        grad = u_apply(spec_sym, p.sigma, x - xbar) / p.gamma
        xt = np.maximum(0.0, x - tau * (grad + psi(v, bases, p.nlevel)))
        vt = v + psi_adjoint(2.0 * xt - x, bases, p.nlevel)
        v = project_l2inf(vt, p.lam)
        x = xt
    return x, v


def project_l2inf(vt, lam):
    """Projection onto the l2,inf ball of radius lam (groups over bands, axis 1):
    v_g = vt_g min(1, lam / ||vt_g||_2).  By Moreau's identity this is the prox of
    the convex conjugate of lam ||.||_{2,1} (Eq. 9's norm)."""
    nrm = np.sqrt((vt ** 2).sum(axis=1, keepdims=True))
    scale = np.where(nrm > lam, lam / np.maximum(nrm, 1e-300), 1.0)
    return vt * scale


# ------------------------------------------------------------------ one pfb step (Eqs. 6-7)
def step(uvw, freq, band_of_chan, wgt, dirty_img, psf_img, wsum_b, x, v, dl, dm, p: Params,
         flags=0, hessian_fn=None):
    """One preconditioned forward-backward step.

      wbar = mean_b wsum_b      (one scalar: I^d, I^psf and the Hessian are divided by it)
      IR   = I^d - H x_k        (one Hessian application = the exact -grad f, Eq. 3;
                                 with p.approx_gradient I^d - I^psf * x_k, Eq. 4)
      delta = CG(U, IR)         (U = I^psf_sym * + sigma Id, Eq. 8)
      xbar = x_k + gamma delta  (Eq. 6)
      x_{k+1}, v = prox(xbar)   (Eq. 7)

    Returns x_{k+1}, v, stats = [objective at x_k up to the data constant,
    relative update, max CG relative residual].  hessian_fn overrides the Hessian
    (tests of the composition at sizes where the direct DFT is too slow)."""
    nband = x.shape[0]
    wbar = float(np.mean(wsum_b))
    if p.approx_gradient:
        # Eq. 4: the PSF convolution (plain, not symmetrised) replaces the Hessian
        hx = psf_conv(np.asarray(psf_img, dtype=np.float64), x) / wbar
    else:
        hx = (hessian(uvw, freq, band_of_chan, wgt, x, dl, dm, flags) if hessian_fn is None
              else hessian_fn(x)) / wbar
    idn = np.asarray(dirty_img, dtype=np.float64) / wbar
    psfn = np.asarray(psf_img, dtype=np.float64) / wbar
    ir = idn - hx
    spec_sym = np.real(psf_spectrum(psfn))
    delta, cgres = cg(spec_sym, p.sigma, ir, p.cg_iters, p.cg_tol)
    xbar = x + p.gamma * delta
    x1, v1 = prox(xbar, v, spec_sym, p)
    bases = basis_list(p.basis_mask)
    fx = 0.5 * float(np.vdot(x, hx)) - float(np.vdot(x, idn))
    obj = fx + p.lam * l21(psi_adjoint(x, bases, p.nlevel))
    nx1 = float(np.linalg.norm(x1))
    rel = float(np.linalg.norm(x1 - x)) / nx1 if nx1 > 0 else 0.0
    return x1, v1, np.array([obj, rel, float(cgres.max()) if nband else 0.0])


# ------------------------------------------------------------------ step-size bound
SAFE_GAMMA_FACTOR = 1.9
BOUND_ITERS = 30


def splitmix64_uniform(n):
    """u_e in [0, 1) for e = 0..n-1 from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
    number generators", OOPSLA 2014) applied to the counter e + 1: the top 53 bits of the mixed word."""
    with np.errstate(over="ignore"):
        z = (np.arange(n, dtype=np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def bound_start(nband, nx, ny):
    """Start vector of the safe-gamma bound: 0.5 + u_e over the flat index of [nband][nx][ny] (a generic
    positive image; a constant one can miss the modes where H exceeds U most)."""
    return 0.5 + splitmix64_uniform(nband * nx * ny).reshape(nband, nx, ny)


def step_bound(uvw, freq, band_of_chan, wgt, psf_img, wsum_b, dl, dm, sigma, iters, cg_iters, z0=None,
               flags=0, hessian_fn=None):
    """Estimate of L_U = lambda_max(U^-1 H) in the step's normalised units (H and the PSF
    divided by wbar = mean_b wsum_b; U = I^psf_sym * + sigma Id, Eq. 8).  Forward-backward
    in the metric U (Eqs. 6-7) converges for gamma < 2 / L_U.  Power iteration on U^-1 H:
        rho_k = z_k^T H z_k / z_k^T U z_k          (generalised Rayleigh quotient, <= L_U)
        z_{k+1} = CG(U, H z_k) / ||CG(U, H z_k)||  (cg_iters iterations per band)
    from z_0 (bound_start, the library's default, when None); returns max_k rho_k."""
    wbar = float(np.mean(wsum_b))
    psfn = np.asarray(psf_img, dtype=np.float64) / wbar
    spec_sym = np.real(psf_spectrum(psfn))
    nband = psfn.shape[0]
    nx, ny = psfn.shape[1] // 2, psfn.shape[2] // 2
    z = bound_start(nband, nx, ny) if z0 is None else np.array(z0, dtype=np.float64)
    best = 0.0
    for _ in range(iters):
        hz = (hessian(uvw, freq, band_of_chan, wgt, z, dl, dm, flags) if hessian_fn is None
              else hessian_fn(z)) / wbar
        rho = float(np.vdot(z, hz)) / float(np.vdot(z, u_apply(spec_sym, sigma, z)))
        best = max(best, rho)
        z, _ = cg(spec_sym, sigma, hz, cg_iters)
        nz = float(np.linalg.norm(z))
        if nz == 0.0:
            break
        z = z / nz
    return best


# ------------------------------------------------------------------ whole solve
def clean(uvw, freq, band_of_chan, vis, wgt, nx, ny, dl, dm, nband, p: Params, max_outer, tol,
          x0=None, v0=None, flags=0):
    """A pfb-clean solve: I^psf on the 2x field and I^d from the data (Eqs. 3-4), then
    preconditioned forward-backward steps (Eqs. 6-7) from x0 (zeros by default) and the
    dual v0, stopping after the first step whose relative update is <= tol (tol <= 0:
    max_outer steps).  n_hessian counts full R^dagger Sigma^-1 R applications: one per
    exact-gradient step and one for I^d and I^psf together (one half each)."""
    psf_img, wsum_b = psf(uvw, freq, band_of_chan, wgt, nx, ny, dl, dm, nband, flags)
    dirty_img, _ = dirty(uvw, freq, band_of_chan, vis, wgt, nx, ny, dl, dm, nband, flags)
    nbasis = len(basis_list(p.basis_mask))
    x = np.zeros((nband, nx, ny)) if x0 is None else np.array(x0, dtype=np.float64)
    v = np.zeros((nbasis, nband, nx, ny)) if v0 is None else np.array(v0, dtype=np.float64)
    hist = []
    n_hessian = 1
    lmax = None
    if p.safe_gamma and not p.approx_gradient:
        # gamma < 2 / L_U is what forward-backward in the metric U needs; the estimate costs
        # BOUND_ITERS Hessian applications, counted
        lmax = step_bound(uvw, freq, band_of_chan, wgt, psf_img, wsum_b, dl, dm, p.sigma, BOUND_ITERS,
                          p.cg_iters, flags=flags)
        n_hessian += BOUND_ITERS
        if lmax > 0:
            p = dataclasses.replace(p, gamma=min(p.gamma, SAFE_GAMMA_FACTOR / lmax))
    while len(hist) < max_outer:
        x, v, st = step(uvw, freq, band_of_chan, wgt, dirty_img, psf_img, wsum_b, x, v, dl, dm, p, flags)
        hist.append(st)
        n_hessian += 0 if p.approx_gradient else 1
        if tol > 0 and st[1] <= tol:
            break
    return {"x": x, "dual": v, "dirty": dirty_img, "psf": psf_img, "wsum": wsum_b, "n_outer": len(hist),
            "n_hessian": n_hessian, "history": np.array(hist).reshape(len(hist), 3), "lmax": lmax,
            "gamma": p.gamma}
