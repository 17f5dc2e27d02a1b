"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
hand-worked values, library routines in special cases, closed forms, invariants
and brute force on tiny inputs (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2101_08072_gb300 import synth

C = synth.C_LIGHT
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _unit_image(nx, ny, i, j, val=1.0, nband=1):
    x = np.zeros((nband, nx, ny))
    x[:, i, j] = val
    return x


# ------------------------------------------------------------------ worked examples
def test_golden_degrid_values():
    g = json.load(open(GOLDEN))
    for case in g["degrid"]:
        x = _unit_image(4, 4, *case["pixel"], val=case["x"])
        uvw = np.array([case["uvw"]], dtype=np.float64)
        v = oracle.degrid(uvw, np.array([C]), np.array([0]), x, 0.6, 0.6)
        assert abs(v[0, 0] - complex(*case["vis"])) < 1e-12, case


def test_golden_grid_values():
    g = json.load(open(GOLDEN))
    for case in g["grid"]:
        uvw = np.array([case["uvw"]], dtype=np.float64)
        vis = np.array([[complex(*case["vis"])]])
        wgt = np.array([[case["wgt"]]])
        img = oracle.grid(uvw, np.array([C]), np.array([0]), vis, wgt, 4, 4, 0.6, 0.6, 1)
        i, j = case["pixel"]
        assert abs(img[0, i, j] - case["image"]) < 1e-12, case


# ------------------------------------------------------------------ R
def test_phase_centre_source_gives_unit_visibilities():
    obs = synth.tiny_observation()
    x = _unit_image(obs.nx, obs.ny, obs.nx // 2, obs.ny // 2)
    v = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    assert np.abs(v - 1.0).max() < 1e-14


def test_degrid_equals_numpy_fft_on_regular_grid():
    """w = 0 and no 1/n: R is a 2-D DFT.  At u = k/(nx dl), v = k'/(ny dm) it equals
    (-1)^(k+k') fft2(x)[k mod nx, k' mod ny] (numpy's forward FFT, minus sign)."""
    rng = np.random.default_rng(7)
    nx, ny, dl = 8, 6, 0.01
    x = rng.normal(size=(1, nx, ny))
    ks, kps = np.meshgrid(np.arange(-nx // 2, nx // 2), np.arange(-ny // 2, ny // 2), indexing="ij")
    ks, kps = ks.ravel(), kps.ravel()
    uvw = np.stack([ks / (nx * dl), kps / (ny * dl), np.zeros_like(ks, dtype=float)], axis=1)
    v = oracle.degrid(uvw, np.array([C]), np.array([0]), x, dl, dl, flags=oracle.NO_DIVIDE_BY_N)[:, 0]
    F = np.fft.fft2(x[0])
    ref = (-1.0) ** (ks + kps) * F[ks % nx, kps % ny]
    assert np.abs(v - ref).max() < 1e-12 * np.abs(F).max()


def test_hermitian_symmetry():
    obs = synth.tiny_observation()
    rng = np.random.default_rng(3)
    x = rng.normal(size=(1, obs.nx, obs.ny))
    v1 = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    v2 = oracle.degrid(-obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    assert np.abs(v2 - np.conj(v1)).max() < 1e-11 * np.abs(v1).max()


def test_shift_theorem_w0():
    """Shifting x by one pixel along l multiplies V by exp(-2 pi i u dl) when w = 0."""
    obs = synth.tiny_observation()
    rng = np.random.default_rng(4)
    x = np.zeros((1, obs.nx, obs.ny))
    x[0, 10:20, 5:30] = rng.normal(size=(10, 25))
    xs = np.roll(x, 1, axis=1)
    f = oracle.NO_DIVIDE_BY_N | oracle.NO_WTERM
    v = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm, flags=f)
    vs = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, xs, obs.dl, obs.dm, flags=f)
    u = obs.uvw[:, 0:1] * obs.freq[None, :] / C
    assert np.abs(vs - v * np.exp(-2j * np.pi * u * obs.dl)).max() < 1e-10 * np.abs(v).max()


def test_linearity_and_row_selection():
    obs = synth.tiny_observation()
    rng = np.random.default_rng(5)
    a, b = rng.normal(size=(2, 1, obs.nx, obs.ny))
    args = (obs.uvw, obs.freq, obs.band_of_chan)
    va = oracle.degrid(*args, a, obs.dl, obs.dm)
    vb = oracle.degrid(*args, b, obs.dl, obs.dm)
    vab = oracle.degrid(*args, 2.0 * a - 3.0 * b, obs.dl, obs.dm)
    assert np.abs(vab - (2 * va - 3 * vb)).max() < 1e-10 * np.abs(vab).max()
    rows = np.array([5, 17, 2000])
    vr = oracle.degrid(*args, a, obs.dl, obs.dm, rows=rows)
    assert np.array_equal(vr, va[rows])


def test_band_mapping():
    """Each channel sees only its own band's image."""
    obs = synth.tiny_observation(nband=2)
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2, obs.nx, obs.ny))
    v = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    x0 = x.copy(); x0[1] = 0
    v0 = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x0, obs.dl, obs.dm)
    b0 = obs.band_of_chan == 0
    assert np.array_equal(v[:, b0], v0[:, b0])
    assert np.abs(v0[:, ~b0]).max() == 0.0


# ------------------------------------------------------------------ R^dagger
def test_adjoint_identity():
    """Re <R x, y> = <x, R^dagger y> with the full w term and 1/n (Eq. 3)."""
    obs = synth.tiny_observation(nband=2)
    rng = np.random.default_rng(8)
    x = rng.normal(size=(2, obs.nx, obs.ny))
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    rx = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    ry = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y, None, obs.nx, obs.ny, obs.dl, obs.dm, 2)
    lhs = float(np.real(np.vdot(rx, y)))
    rhs = float(np.sum(x * ry))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), np.linalg.norm(rx) * np.linalg.norm(y))


def test_grid_equals_numpy_ifft_on_regular_grid():
    rng = np.random.default_rng(9)
    nx, ny, dl = 6, 8, 0.02
    ks, kps = np.meshgrid(np.arange(-nx // 2, nx // 2), np.arange(-ny // 2, ny // 2), indexing="ij")
    ks, kps = ks.ravel(), kps.ravel()
    uvw = np.stack([ks / (nx * dl), kps / (ny * dl), np.zeros(ks.size)], axis=1)
    y = synth.random_vis(rng, (ks.size, 1))
    img = oracle.grid(uvw, np.array([C]), np.array([0]), y, None, nx, ny, dl, dl, 1,
                      flags=oracle.NO_DIVIDE_BY_N)[0]
    Y = np.zeros((nx, ny), dtype=complex)
    Y[ks % nx, kps % ny] = (-1.0) ** (ks + kps) * y[:, 0]
    ref = np.real(np.fft.ifft2(Y)) * nx * ny
    assert np.abs(img - ref).max() < 1e-12 * np.abs(ref).max()


def test_weights_and_pixel_selection():
    obs = synth.tiny_observation()
    rng = np.random.default_rng(10)
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    a = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y, w, obs.nx, obs.ny, obs.dl, obs.dm, 1)
    b = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y * w, None, obs.nx, obs.ny, obs.dl, obs.dm, 1)
    assert np.abs(a - b).max() < 1e-10 * np.abs(a).max()
    pix = np.array([0, 77, 4095])
    s = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y, w, obs.nx, obs.ny, obs.dl, obs.dm, 1, pix=pix)
    assert np.array_equal(s, a.reshape(-1)[pix])


def test_dense_matrix_brute_force():
    """Columns of R from unit images and rows of R^dagger from unit visibilities:
    the two matrices are transposes under the real inner product."""
    obs = synth.tiny_observation(nx=8, ny=8, ntime=3, n_ant=5, nchan=2)
    npx = obs.nx * obs.ny
    Rm = np.zeros((obs.nvis, npx), dtype=complex)
    for p in range(npx):
        e = np.zeros((1, obs.nx, obs.ny)); e.reshape(-1)[p] = 1.0
        Rm[:, p] = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, e, obs.dl, obs.dm).reshape(-1)
    Ra = np.zeros((npx, obs.nvis, 2))
    for k in range(obs.nvis):
        for part, val in ((0, 1.0), (1, 1.0j)):
            y = np.zeros(obs.nvis, dtype=complex); y[k] = val
            Ra[:, k, part] = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y.reshape(obs.nrow, obs.nchan),
                                         None, obs.nx, obs.ny, obs.dl, obs.dm, 1).reshape(-1)
    # Re <R e_p, e_k> = Re R[k,p];  Re <R e_p, i e_k> = Im R[k,p]
    assert np.abs(Ra[:, :, 0] - Rm.real.T).max() < 1e-12
    assert np.abs(Ra[:, :, 1] - Rm.imag.T).max() < 1e-12


# ------------------------------------------------------------------ I^d, PSF, H
def test_dirty_of_centre_source_is_psf_crop():
    obs = synth.tiny_observation()
    rng = np.random.default_rng(11)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    x = _unit_image(obs.nx, obs.ny, obs.nx // 2, obs.ny // 2)
    v = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    d, ws = oracle.dirty(obs.uvw, obs.freq, obs.band_of_chan, v, w, obs.nx, obs.ny, obs.dl, obs.dm, 1)
    p, ws2 = oracle.psf(obs.uvw, obs.freq, obs.band_of_chan, w, obs.nx, obs.ny, obs.dl, obs.dm, 1)
    h = obs.nx // 2
    crop = p[:, h:h + obs.nx, h:h + obs.ny]
    assert np.abs(d - crop).max() < 1e-10 * ws[0]
    assert abs(p[0, obs.nx, obs.ny] - w.sum()) < 1e-10 * w.sum()
    assert np.allclose(ws, [w.sum()]) and np.allclose(ws2, ws)
    assert p[0, obs.nx, obs.ny] == pytest.approx(p.max(), rel=1e-12)


def test_psf_point_symmetric_at_w0():
    obs = synth.tiny_observation(nx=16, ny=16)
    uvw = obs.uvw.copy(); uvw[:, 2] = 0.0
    p, _ = oracle.psf(uvw, obs.freq, obs.band_of_chan, None, obs.nx, obs.ny, obs.dl, obs.dm, 1)
    n = obs.nx
    a = p[0, 1:, 1:]
    assert np.abs(a - a[::-1, ::-1]).max() < 1e-10 * p.max()
    # with w != 0 the symmetry is broken (the n-1 term)
    p2, _ = oracle.psf(obs.uvw * 50.0, obs.freq, obs.band_of_chan, None, n, n, obs.dl * 20, obs.dm * 20, 1)
    b = p2[0, 1:, 1:]
    assert np.abs(b - b[::-1, ::-1]).max() > 1e-6 * p2.max()


def test_hessian_equals_psf_conv_at_w0():
    obs = synth.tiny_observation(nx=16, ny=16)
    uvw = obs.uvw.copy(); uvw[:, 2] = 0.0
    rng = np.random.default_rng(12)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    x = rng.normal(size=(1, obs.nx, obs.ny))
    a = (uvw, obs.freq, obs.band_of_chan)
    f = oracle.NO_DIVIDE_BY_N
    hx = oracle.hessian(*a, w, x, obs.dl, obs.dm, flags=f)
    p, _ = oracle.psf(*a, w, obs.nx, obs.ny, obs.dl, obs.dm, 1, flags=f)
    assert np.abs(hx - oracle.psf_conv_direct(p, x)).max() < 1e-10 * np.abs(hx).max()
    # with 1/n: H x = n^-1 (PSF_raw * (n^-1 x))
    l = (np.arange(obs.nx) - obs.nx // 2) * obs.dl
    m = (np.arange(obs.ny) - obs.ny // 2) * obs.dm
    ninv = 1.0 / np.sqrt(1.0 - l[:, None] ** 2 - m[None, :] ** 2)
    hx2 = oracle.hessian(*a, w, x, obs.dl, obs.dm)
    ref = ninv * oracle.psf_conv_direct(p, ninv * x)
    assert np.abs(hx2 - ref).max() < 1e-10 * np.abs(hx2).max()


def test_hessian_differs_from_psf_conv_when_noncoplanar():
    """Eq. 4 neglects the w term: with w != 0 the PSF convolution is only approximate."""
    obs = synth.tiny_observation(nx=16, ny=16)
    rng = np.random.default_rng(13)
    uvw = obs.uvw * 50.0
    dl = obs.dl * 20
    x = rng.uniform(0, 1, (1, 16, 16))
    hx = oracle.hessian(uvw, obs.freq, obs.band_of_chan, None, x, dl, dl)
    p, _ = oracle.psf(uvw, obs.freq, obs.band_of_chan, None, 16, 16, dl, dl, 1)
    rel = np.linalg.norm(hx - oracle.psf_conv(p, x)) / np.linalg.norm(hx)
    assert rel > 1e-3


def test_hessian_symmetric_psd():
    obs = synth.tiny_observation(nx=16, ny=16)
    rng = np.random.default_rng(14)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    x, z = rng.normal(size=(2, 1, 16, 16))
    a = (obs.uvw, obs.freq, obs.band_of_chan, w)
    hx = oracle.hessian(*a, x, obs.dl, obs.dm)
    hz = oracle.hessian(*a, z, obs.dl, obs.dm)
    assert abs(np.sum(hx * z) - np.sum(x * hz)) < 1e-10 * abs(np.sum(hx * z))
    rx = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    assert np.sum(x * hx) == pytest.approx(np.sum(w * np.abs(rx) ** 2), rel=1e-11)


# ------------------------------------------------------------------ gradient (Eqs. 2-3)
def test_gradient_central_differences_and_zero_at_truth():
    obs = synth.tiny_observation(nx=16, ny=16)
    rng = np.random.default_rng(15)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    xt = synth.sparse_random_image(rng, 1, 16, 16, 0.1)
    V = oracle.degrid(*a, xt, obs.dl, obs.dm)
    d, _ = oracle.dirty(*a, V, w, 16, 16, obs.dl, obs.dm, 1)
    g_true = oracle.hessian(*a, w, xt, obs.dl, obs.dm) - d
    assert np.abs(g_true).max() < 1e-10 * np.abs(d).max()
    V = V + synth.complex_noise(rng, V.shape)
    d, _ = oracle.dirty(*a, V, w, 16, 16, obs.dl, obs.dm, 1)
    x = rng.uniform(0, 1, (1, 16, 16))
    g = oracle.hessian(*a, w, x, obs.dl, obs.dm) - d

    def f(xx):
        r = V - oracle.degrid(*a, xx, obs.dl, obs.dm)
        return 0.5 * float(np.sum(w * np.abs(r) ** 2))

    for p in rng.choice(256, 6, replace=False):
        e = np.zeros_like(x); e.reshape(-1)[p] = 0.5
        fd = (f(x + e) - f(x - e)) / 1.0
        assert fd == pytest.approx(g.reshape(-1)[p], rel=1e-7, abs=1e-9 * np.abs(g).max())


# ------------------------------------------------------------------ PSF convolution
def test_psf_conv_fft_equals_direct_sum():
    rng = np.random.default_rng(16)
    psf = rng.normal(size=(2, 24, 20))
    x = rng.normal(size=(2, 12, 10))
    a = oracle.psf_conv_direct(psf, x)
    b = oracle.psf_conv(psf, x)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_psf_conv_delta_is_identity_and_shift():
    x = np.random.default_rng(17).normal(size=(1, 8, 8))
    d = np.zeros((1, 16, 16)); d[0, 8, 8] = 1.0
    assert np.abs(oracle.psf_conv_direct(d, x) - x).max() == 0.0
    d2 = np.zeros((1, 16, 16)); d2[0, 9, 8] = 1.0      # centre + one pixel along l
    y = oracle.psf_conv_direct(d2, x)
    assert np.abs(y[0, 1:] - x[0, :-1]).max() == 0.0 and np.abs(y[0, 0]).max() == 0.0


# ------------------------------------------------------------------ CG on U (Eq. 8)
def _test_psf(nx, ny, seed=18):
    obs = synth.tiny_observation(nx=nx, ny=ny, seed=seed)
    p, ws = oracle.psf(obs.uvw, obs.freq, obs.band_of_chan, None, nx, ny, obs.dl, obs.dm, 1)
    return p / ws[0]


def test_cg_matches_dense_solve():
    nx = ny = 8
    p = _test_psf(nx, ny)
    spec = np.real(oracle.psf_spectrum(p))
    sigma = 0.05
    n = nx * ny
    U = np.zeros((n, n))
    for k in range(n):
        e = np.zeros((1, nx, ny)); e.reshape(-1)[k] = 1.0
        U[:, k] = oracle.u_apply(spec, sigma, e).reshape(-1)
    assert np.abs(U - U.T).max() < 1e-12                     # symmetric by construction
    assert np.linalg.eigvalsh(U).min() > 0
    b = np.random.default_rng(19).normal(size=(1, nx, ny))
    delta, res = oracle.cg(spec, sigma, b, iters=200, tol=1e-13)
    ref = np.linalg.solve(U, b.reshape(-1)).reshape(1, nx, ny)
    assert np.abs(delta - ref).max() < 1e-9 * np.abs(ref).max()
    assert res[0] < 1e-12


def test_cg_iterates_minimise_over_krylov_spaces():
    """CG at a fixed, unconverged iteration count k: its iterate is the minimiser of the U-norm error
    (delta - U^-1 b)^T U (delta - U^-1 b) over the Krylov space span{b, U b, ..., U^(k-1) b} (Hestenes
    and Stiefel 1952).  The minimiser is computed here from an orthonormal basis Q of that space:
    delta_k = Q (Q^T U Q)^-1 Q^T b.  Also the reported relative residual ||b - U delta_k|| / ||b||."""
    nx = ny = 8
    p = _test_psf(nx, ny)
    spec = np.real(oracle.psf_spectrum(p))
    sigma = 0.05
    n = nx * ny
    U = np.zeros((n, n))
    for k in range(n):
        e = np.zeros((1, nx, ny)); e.reshape(-1)[k] = 1.0
        U[:, k] = oracle.u_apply(spec, sigma, e).reshape(-1)
    b = np.random.default_rng(27).normal(size=(1, nx, ny))
    bv = b.reshape(-1)
    for k in (1, 2, 3, 5):
        delta, res = oracle.cg(spec, sigma, b, iters=k, tol=0.0)
        K = np.stack([np.linalg.matrix_power(U, m) @ bv for m in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        ref = Q @ np.linalg.solve(Q.T @ U @ Q, Q.T @ bv)
        assert np.abs(delta.reshape(-1) - ref).max() <= 1e-9 * np.abs(ref).max(), k
        assert res[0] == pytest.approx(np.linalg.norm(bv - U @ ref) / np.linalg.norm(bv), rel=1e-7), k


def test_symmetrised_psf_operator_is_symmetric_part():
    """U uses Re(spectrum): the convolution with the PSF symmetrised about its
    centre, i.e. (M + M^T)/2 for M the PSF-convolution matrix."""
    nx = ny = 6
    rng = np.random.default_rng(20)
    p = rng.normal(size=(1, 12, 12))
    n = nx * ny
    M = np.zeros((n, n)); S = np.zeros((n, n))
    spec = np.real(oracle.psf_spectrum(p))
    for k in range(n):
        e = np.zeros((1, nx, ny)); e.reshape(-1)[k] = 1.0
        M[:, k] = oracle.psf_conv_direct(p, e).reshape(-1)
        S[:, k] = oracle.u_apply(spec, 0.0, e).reshape(-1)
    assert np.abs(S - 0.5 * (M + M.T)).max() < 1e-12


# ------------------------------------------------------------------ wavelets (Eq. 9's Psi)
def test_daubechies_filter_conditions():
    for N in range(1, 7):
        h = oracle.daubechies(N)
        assert h.shape == (2 * N,)
        assert h.sum() == pytest.approx(math.sqrt(2.0), abs=1e-13)
        for m in range(N):
            s = float(np.dot(h[: 2 * N - 2 * m], h[2 * m:]))
            assert s == pytest.approx(1.0 if m == 0 else 0.0, abs=1e-12)
        k = np.arange(2 * N)
        for pw in range(N):
            assert abs(float(np.sum((-1.0) ** k * k ** pw * h))) < 1e-9 * max(1, (2 * N) ** pw)
    s3 = math.sqrt(3.0)
    db2 = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2.0))
    assert np.abs(oracle.daubechies(2) - db2).max() < 1e-14


def test_dwt_orthonormal_and_haar_closed_form():
    rng = np.random.default_rng(21)
    img = rng.normal(size=(16, 8))
    for N in (1, 3, 6):
        h = oracle.daubechies(N)
        c = oracle.dwt2(img, h, 3)
        assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(img), rel=1e-13)
        assert np.abs(oracle.idwt2(c, h, 3) - img).max() < 1e-12
    c = oracle.dwt2(np.full((4, 4), 3.0), oracle.daubechies(1), 1)
    ref = np.zeros((4, 4)); ref[:2, :2] = 6.0
    assert np.abs(c - ref).max() < 1e-14


def _dwt_constant_failures(dwt2_fn):
    """Failures of the multi-level DWT on constant images (Eq. 9's Psi_k, Mallat layout).
    A constant c has zero detail at every level (the high-pass filter sums to 0, the
    first vanishing moment) and a low-pass output of sqrt(2) c per axis and level, so
    after L levels of the 2-D transform only the coarsest approximation block
    [0:n/2^L, 0:m/2^L] is non-zero and it holds c 2^L.  A recursion on the wrong
    quadrant, a wrong block size or a skipped level breaks this."""
    bad = []
    c0 = 1.7
    for N in range(1, 7):
        h = oracle.daubechies(N)
        for L in (1, 2, 3):
            img = np.full((16, 32), c0)
            got = dwt2_fn(img, h, L)
            ref = np.zeros_like(img)
            ref[: 16 >> L, : 32 >> L] = c0 * 2.0 ** L
            err = float(np.abs(got - ref).max())
            if err > 1e-12:
                bad.append((N, L, err))
    return bad


def _haar_two_level_expected():
    """Two levels of the 2-D Haar DWT of the separable 8 x 8 image x = a b^T, worked by
    hand.  One 1-D Haar level maps x to ((x0+x1), (x2+x3), ... | (x0-x1), (x2-x3), ...)/sqrt2.
      a = [1..8]:              level 1 A1 = [3, 7, 11, 15]/sqrt2, D1 = [-1, -1, -1, -1]/sqrt2
                               level 2 (on A1) A2 = [10, 26]/2 = [5, 13], D2 = [-4, -4]/2 = [-2, -2]
      b = [1,0,0,2,3,1,0,1]:   level 1 A1 = [1, 2, 4, 1]/sqrt2, D1 = [1, -2, 2, -1]/sqrt2
                               level 2 A2 = [3, 5]/2, D2 = [-1, 3]/2
    A 2-D level on a separable block gives the four outer products of the 1-D halves, and
    the second level transforms only the approximation block [0:4, 0:4]."""
    r2 = math.sqrt(2.0)
    a_A1, a_D1 = np.array([3, 7, 11, 15]) / r2, np.array([-1, -1, -1, -1]) / r2
    a_A2, a_D2 = np.array([5.0, 13.0]), np.array([-2.0, -2.0])
    b_A1, b_D1 = np.array([1, 2, 4, 1]) / r2, np.array([1, -2, 2, -1]) / r2
    b_A2, b_D2 = np.array([1.5, 2.5]), np.array([-0.5, 1.5])
    c = np.zeros((8, 8))
    c[0:2, 0:2] = np.outer(a_A2, b_A2)
    c[0:2, 2:4] = np.outer(a_A2, b_D2)
    c[2:4, 0:2] = np.outer(a_D2, b_A2)
    c[2:4, 2:4] = np.outer(a_D2, b_D2)
    c[0:4, 4:8] = np.outer(a_A1, b_D1)
    c[4:8, 0:4] = np.outer(a_D1, b_A1)
    c[4:8, 4:8] = np.outer(a_D1, b_D1)
    return np.outer(np.arange(1.0, 9.0), [1, 0, 0, 2, 3, 1, 0, 1]), c


def _wrong_quadrant_dwt2(img, h, nlevel):
    """A planted mistake: the recursion continues on the detail block [n/2:n, 0:m/2]
    instead of the approximation block [0:n/2, 0:m/2]."""
    c = np.array(img, dtype=np.float64)
    g = oracle.highpass(h)
    r0, n, m = 0, c.shape[0], c.shape[1]
    for _ in range(nlevel):
        blk = oracle._dwt1(c[r0:r0 + n, :m], h, g, 0)
        c[r0:r0 + n, :m] = oracle._dwt1(blk, h, g, 1)
        r0, n, m = r0 + n // 2, n // 2, m // 2
    return c


def test_dwt_multilevel_recursion_constant_images():
    assert _dwt_constant_failures(oracle.dwt2) == []
    # the pin rejects a recursion on the wrong quadrant (planted, CPU only)
    assert len(_dwt_constant_failures(_wrong_quadrant_dwt2)) > 0


def test_dwt_two_level_haar_hand_worked():
    x, ref = _haar_two_level_expected()
    assert np.abs(oracle.dwt2(x, oracle.daubechies(1), 2) - ref).max() < 1e-13
    assert np.abs(oracle.idwt2(ref, oracle.daubechies(1), 2) - x).max() < 1e-13
    assert np.abs(_wrong_quadrant_dwt2(x, oracle.daubechies(1), 2) - ref).max() > 0.1


def test_psi_tight_frame():
    rng = np.random.default_rng(22)
    x = rng.normal(size=(2, 16, 16))
    bases = oracle.basis_list(0b1111111)
    c = oracle.psi_adjoint(x, bases, 2)
    assert np.abs(oracle.psi(c, bases, 2) - x).max() < 1e-12           # Psi Psi^dagger = Id
    assert np.linalg.norm(c) == pytest.approx(np.linalg.norm(x), rel=1e-12)


# ------------------------------------------------------------------ prox (Eq. 7)
def test_prox_closed_form_sigma_metric_dirac():
    """PSF = 0 so U = sigma Id, Psi = Dirac: Eq. 7 has the closed form
    x_g = max(xbar_g, 0) * max(0, 1 - gamma lam / (sigma ||max(xbar_g, 0)||_2))."""
    rng = np.random.default_rng(23)
    nb, nx, ny = 3, 8, 8
    xbar = rng.normal(size=(nb, nx, ny))
    spec0 = np.zeros((nb, 16, 16))
    p = oracle.Params(gamma=0.7, sigma=2.0, lam=0.9, pd_iters=3000, basis_mask=1)
    x, v = oracle.prox(xbar, np.zeros((1, nb, nx, ny)), spec0, p)
    z = np.maximum(xbar, 0)
    nrm = np.sqrt((z ** 2).sum(axis=0, keepdims=True))
    ref = z * np.maximum(0.0, 1.0 - p.gamma * p.lam / (p.sigma * np.maximum(nrm, 1e-300)))
    assert np.abs(x - ref).max() < 1e-8


def test_prox_lambda0_kkt():
    nx = ny = 8
    pn = _test_psf(nx, ny)
    spec = np.real(oracle.psf_spectrum(pn))
    rng = np.random.default_rng(24)
    xbar = rng.normal(size=(1, nx, ny)) * 0.1
    p = oracle.Params(gamma=1.0, sigma=0.05, lam=0.0, pd_iters=4000)
    x, _ = oracle.prox(xbar, np.zeros((1, 1, nx, ny)), spec, p)
    g = oracle.u_apply(spec, p.sigma, x - xbar)
    assert x.min() >= 0
    assert g.min() > -1e-7
    assert np.abs(x * g).max() < 1e-7


def _prox_kkt(x, v, xbar, spec, p):
    """Optimality of Eq. 7 with r of Eq. 9 at (x, v): x is the minimiser of
    lam ||Psi^dagger x||_{2,1} + iota_+(x) + (1/2 gamma)(x - xbar)^T U (x - xbar) and v a
    dual certificate when
      x >= 0;  ||v_g|| <= lam for every group g (bands of one basis coefficient);
      v_g = lam c_g / ||c_g|| wherever c_g = (Psi^dagger x)_g != 0  (v in lam d||.||_{2,1}(c));
      g = U (x - xbar) / gamma + Psi v >= 0 and x . g = 0  (-g in the normal cone of x >= 0).
    Returns the largest violation of each condition, scaled by lam or |g|."""
    bases = oracle.basis_list(p.basis_mask)
    c = oracle.psi_adjoint(x, bases, p.nlevel)
    cn = np.sqrt((c ** 2).sum(axis=1, keepdims=True))
    vn = np.sqrt((v ** 2).sum(axis=1))
    act = np.broadcast_to(cn > 1e-9, v.shape)
    dirn = np.abs(v - p.lam * c / np.maximum(cn, 1e-300))[act]
    g = oracle.u_apply(spec, p.sigma, x - xbar) / p.gamma + oracle.psi(v, bases, p.nlevel)
    return {"neg_x": float(max(0.0, -x.min())),
            "ball": float(max(0.0, vn.max() - p.lam)) / p.lam,
            "subgrad": float(dirn.max()) / p.lam if dirn.size else 0.0,
            "neg_g": float(max(0.0, -g.min())),
            "compl": float(np.abs(x * g).max())}


def _kkt_case():
    nx = ny = 8
    spec1 = np.real(oracle.psf_spectrum(_test_psf(nx, ny)))
    spec = 0.3 * np.concatenate([spec1, 0.5 * spec1])     # two bands, U = PSF_sym* + sigma Id
    xbar = np.random.default_rng(25).normal(size=(2, nx, ny))
    p = oracle.Params(gamma=1.0, sigma=1.0, lam=0.2, pd_iters=400, basis_mask=0b1111111, nlevel=2)
    return xbar, spec, p


def test_prox_lambda_positive_kkt_full_dictionary():
    """The converged Condat-Vu prox (lam > 0, full Dirac + db1..db6 dictionary, U metric)
    satisfies the optimality conditions of Eq. 7; a planted projection radius of 2 lam
    or lam / 2 in the dual update (CPU only) violates them."""
    xbar, spec, p = _kkt_case()
    nb = xbar.shape[0]
    x, v = oracle.prox(xbar, np.zeros((7, nb) + xbar.shape[1:]), spec, p)
    k = _prox_kkt(x, v, xbar, spec, p)
    assert k["neg_x"] == 0.0
    assert k["ball"] < 1e-12 and k["subgrad"] < 1e-6, k
    assert k["neg_g"] < 1e-9 and k["compl"] < 1e-9, k
    assert 0.2 < float((x > 0).mean()) < 0.8          # both sides of the positivity constraint occur
    proj = oracle.project_l2inf
    for wrong in (2.0, 0.5):
        try:
            oracle.project_l2inf = lambda vt, lam, f=wrong: proj(vt, f * lam)
            xw, vw = oracle.prox(xbar, np.zeros((7, nb) + xbar.shape[1:]), spec, p)
        finally:
            oracle.project_l2inf = proj
        kw = _prox_kkt(xw, vw, xbar, spec, p)
        assert max(kw["ball"], kw["subgrad"]) > 0.1, (wrong, kw)


# ------------------------------------------------------------------ step (Eqs. 6-7)
def test_step_fixed_point_at_truth():
    """Noiseless data, lam = 0: the true non-negative image makes the exact residual
    vanish (Eq. 3), so CG returns 0 and the prox of a feasible point with lam = 0 is
    the point itself: x_true is a fixed point of one step."""
    obs = synth.tiny_observation(nx=16, ny=16)
    rng = np.random.default_rng(25)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    xt = synth.sparse_random_image(rng, 1, 16, 16, 0.2)
    V = oracle.degrid(*a, xt, obs.dl, obs.dm)
    d, ws = oracle.dirty(*a, V, w, 16, 16, obs.dl, obs.dm, 1)
    p, _ = oracle.psf(*a, w, 16, 16, obs.dl, obs.dm, 1)
    prm = oracle.Params(gamma=1.0, sigma=1e-2, lam=0.0, cg_iters=20, pd_iters=50)
    x1, v1, st = oracle.step(*a, w, d, p, ws, xt, np.zeros((1, 1, 16, 16)), obs.dl, obs.dm, prm)
    assert np.abs(x1 - xt).max() < 1e-9
    assert st[1] < 1e-9


def test_step_equals_dense_preconditioned_step():
    """lam = 0 and an iterate well inside the positive orthant: the prox of Eq. 7 is the identity and
    the dual stays 0, so a step with CG run to convergence is x + gamma U^-1 (I^d - H x) / wbar
    (Eqs. 6-8).  Built here from dense matrices: H column by column from the Hessian of unit images,
    U = (M + M^T) / 2 + sigma Id with M[(i,j),(i',j')] = I^psf[i - i' + nx, j - j' + ny] / wbar (the
    linear PSF convolution, symmetrised), solved by numpy.  The statistics follow the same formulas:
    objective x.Hx / (2 wbar) - x.I^d / wbar and relative update ||x1 - x|| / ||x1||."""
    nx = ny = 8
    obs = synth.tiny_observation(nx=nx, ny=ny)
    rng = np.random.default_rng(28)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    xt = synth.point_source_image(rng, 1, nx, ny, 4)
    V = oracle.degrid(*a, xt, obs.dl, obs.dm) + synth.complex_noise(rng, (obs.nrow, obs.nchan), 1e-2)
    d, ws = oracle.dirty(*a, V, w, nx, ny, obs.dl, obs.dm, 1)
    p, _ = oracle.psf(*a, w, nx, ny, obs.dl, obs.dm, 1)
    x0 = 2.0 + rng.uniform(0.0, 1.0, (1, nx, ny))
    gamma, sigma = 0.5, 0.3
    prm = oracle.Params(gamma=gamma, sigma=sigma, lam=0.0, cg_iters=100, pd_iters=5)
    x1, v1, st = oracle.step(*a, w, d, p, ws, x0, np.zeros((1, 1, nx, ny)), obs.dl, obs.dm, prm)
    # dense H and U
    n = nx * ny
    wbar = float(np.mean(ws))
    Hd = np.zeros((n, n))
    M = np.zeros((n, n))
    for k in range(n):
        i, j = divmod(k, ny)
        Hd[:, k] = oracle.hessian(*a, w, _unit_image(nx, ny, i, j), obs.dl, obs.dm).ravel()
        for k2 in range(n):
            i2, j2 = divmod(k2, ny)
            M[k2, k] = p[0, i2 - i + nx, j2 - j + ny]
    U = 0.5 * (M + M.T) / wbar + sigma * np.eye(n)
    xv = x0.ravel()
    ir = (d.ravel() - Hd @ xv) / wbar
    xbar = xv + gamma * np.linalg.solve(U, ir)
    assert xbar.min() > 0.1   # the prox is the identity there
    assert np.abs(x1.ravel() - xbar).max() <= 1e-9 * np.abs(xbar).max()
    assert np.abs(v1).max() == 0.0
    obj = 0.5 * xv @ (Hd @ xv) / wbar - xv @ d.ravel() / wbar
    assert st[0] == pytest.approx(obj, rel=1e-10)
    assert st[1] == pytest.approx(np.linalg.norm(xbar - xv) / np.linalg.norm(xbar), rel=1e-9)
    assert st[2] < 1e-8


def _dense_h_u(nx, ny, w, obs, p, ws, sigma):
    """Dense normalised H / wbar and U = PSF_sym / wbar + sigma Id of a one-band tiny problem, built column
    by column from unit images (H) and from the PSF samples (U), independent of the power iteration."""
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    n = nx * ny
    wbar = float(np.mean(ws))
    Hd = np.zeros((n, n))
    M = np.zeros((n, n))
    for k in range(n):
        i, j = divmod(k, ny)
        Hd[:, k] = oracle.hessian(*a, w, _unit_image(nx, ny, i, j), obs.dl, obs.dm).ravel()
        for k2 in range(n):
            i2, j2 = divmod(k2, ny)
            M[k2, k] = p[0, i2 - i + nx, j2 - j + ny]
    return Hd / wbar, 0.5 * (M + M.T) / wbar + sigma * np.eye(n)


def test_step_bound_is_generalised_eigenvalue():
    """L_U = lambda_max(U^-1 H) (the bound gamma < 2 / L_U of forward-backward in the metric U,
    Eqs. 6-8): the power iteration's Rayleigh quotients never exceed the largest eigenvalue of the
    dense generalised problem H z = lambda U z, and converge to it (slowly: the gap to the second
    eigenvalue is small, 60 iterations come within 1e-4)."""
    import scipy.linalg
    nx = ny = 8
    obs = synth.tiny_observation(nx=nx, ny=ny)
    rng = np.random.default_rng(29)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    p, ws = oracle.psf(*a, w, nx, ny, obs.dl, obs.dm, 1)
    sigma = 0.05
    Hn, U = _dense_h_u(nx, ny, w, obs, p, ws, sigma)
    lam = scipy.linalg.eigh(Hn, U, eigvals_only=True)
    lmax = float(lam[-1])
    est = [oracle.step_bound(*a, w, p, ws, obs.dl, obs.dm, sigma, k, cg_iters=300) for k in (1, 3, 60)]
    assert all(e <= lmax * (1 + 1e-10) for e in est)
    assert est[0] <= est[1] <= est[2]
    assert est[2] == pytest.approx(lmax, rel=2e-4)


def test_bound_start_is_splitmix64():
    """The start vector of the safe-gamma bound: 0.5 + u_e with u_e the top 53 bits of SplitMix64 of
    e + 1.  The first word is the generator's published first output from seed 0, 0xE220A8397B1DCDAF."""
    u = oracle.splitmix64_uniform(4)
    assert u[0] == (0xE220A8397B1DCDAF >> 11) * 2.0 ** -53
    assert np.all((u >= 0) & (u < 1)) and len(set(u.tolist())) == 4
    z = oracle.bound_start(2, 4, 4)
    assert z.shape == (2, 4, 4) and z.flat[0] == 0.5 + u[0]


def test_clean_safe_gamma_caps_the_step():
    """With safe_gamma the solve takes gamma = min(gamma, 1.9 / L_U) and counts the bound's Hessians:
    the same as a plain solve run with that gamma."""
    nx = ny = 8
    obs = synth.tiny_observation(nx=nx, ny=ny)
    rng = np.random.default_rng(30)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    xt = synth.point_source_image(rng, 1, nx, ny, 3)
    V = oracle.degrid(*a, xt, obs.dl, obs.dm) + synth.complex_noise(rng, (obs.nrow, obs.nchan), 1e-3)
    prm = oracle.Params(gamma=3.0, sigma=0.05, lam=1e-3, cg_iters=20, pd_iters=10, safe_gamma=True)
    r = oracle.clean(*a, V, w, nx, ny, obs.dl, obs.dm, 1, prm, max_outer=3, tol=0.0)
    assert r["lmax"] > 0 and r["gamma"] == pytest.approx(oracle.SAFE_GAMMA_FACTOR / r["lmax"])
    assert r["gamma"] < 3.0 and r["n_hessian"] == 1 + oracle.BOUND_ITERS + 3
    p2 = oracle.Params(gamma=r["gamma"], sigma=0.05, lam=1e-3, cg_iters=20, pd_iters=10)
    r2 = oracle.clean(*a, V, w, nx, ny, obs.dl, obs.dm, 1, p2, max_outer=3, tol=0.0)
    assert np.abs(r["x"] - r2["x"]).max() <= 1e-12 * max(np.abs(r2["x"]).max(), 1e-30)


def test_step_decreases_objective():
    obs = synth.tiny_observation(nx=16, ny=16)
    rng = np.random.default_rng(26)
    w = np.ones((obs.nrow, obs.nchan))
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    xt = synth.point_source_image(rng, 1, 16, 16, 5)
    V = oracle.degrid(*a, xt, obs.dl, obs.dm) + synth.complex_noise(rng, (obs.nrow, obs.nchan))
    d, ws = oracle.dirty(*a, V, w, 16, 16, obs.dl, obs.dm, 1)
    p, _ = oracle.psf(*a, w, 16, 16, obs.dl, obs.dm, 1)
    prm = oracle.Params(gamma=1.0, sigma=1e-2, lam=1e-3, cg_iters=30, pd_iters=100)
    x = np.zeros((1, 16, 16)); v = np.zeros((1, 1, 16, 16))
    objs = []
    for _ in range(4):
        x, v, st = oracle.step(*a, w, d, p, ws, x, v, obs.dl, obs.dm, prm)
        objs.append(st[0])
    assert x.min() >= 0
    assert objs[-1] < objs[0]


# ------------------------------------------------------------------ approximate gradient (Eq. 4)
def test_approx_gradient_step_equals_exact_at_w0():
    """For a coplanar array (w = 0) without the 1/n factor the Hessian is exactly the
    PSF convolution, so the step with the approximate gradient of Eq. 4 must equal
    the exact-gradient step: a wrong normalisation, sign or PSF orientation in the
    Eq. 4 branch breaks this."""
    obs = synth.tiny_observation(nx=16, ny=16)
    uvw = obs.uvw.copy(); uvw[:, 2] = 0.0
    rng = np.random.default_rng(41)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    a = (uvw, obs.freq, obs.band_of_chan)
    f = oracle.NO_DIVIDE_BY_N
    xt = synth.point_source_image(rng, 1, 16, 16, 4)
    V = oracle.degrid(*a, xt, obs.dl, obs.dm, flags=f) + synth.complex_noise(rng, (obs.nrow, obs.nchan), 1e-3)
    d, ws = oracle.dirty(*a, V, w, 16, 16, obs.dl, obs.dm, 1, flags=f)
    p, _ = oracle.psf(*a, w, 16, 16, obs.dl, obs.dm, 1, flags=f)
    x0 = 0.3 * xt
    v0 = np.zeros((1, 1, 16, 16))
    prm = oracle.Params(gamma=1.0, sigma=1e-2, lam=1e-3, cg_iters=10, pd_iters=20)
    xe, ve, se = oracle.step(*a, w, d, p, ws, x0, v0, obs.dl, obs.dm, prm, f)
    prm.approx_gradient = True
    xa, va, sa = oracle.step(*a, w, d, p, ws, x0, v0, obs.dl, obs.dm, prm, f)
    assert np.abs(xa - xe).max() < 1e-10 * np.abs(xe).max()
    assert np.abs(va - ve).max() < 1e-10 * max(np.abs(ve).max(), 1e-30) + 1e-15
    assert sa[0] == pytest.approx(se[0], rel=1e-10)


def test_approx_gradient_error_grows_with_field():
    """The wide-field error of Eq. 4: ||H x - I^psf * x|| / ||H x|| vanishes (to
    rounding) for a coplanar array without 1/n and grows with the field of view as
    the w (n - 1) phase grows."""
    obs = synth.tiny_observation(nx=16, ny=16)
    rng = np.random.default_rng(42)
    x = rng.uniform(0, 1, (1, 16, 16))
    uvw = obs.uvw

    def err(dl, flags=0, coplanar=False):
        u = uvw.copy()
        if coplanar:
            u[:, 2] = 0.0
        hx = oracle.hessian(u, obs.freq, obs.band_of_chan, None, x, dl, dl, flags=flags)
        p, _ = oracle.psf(u, obs.freq, obs.band_of_chan, None, 16, 16, dl, dl, 1, flags=flags)
        return np.linalg.norm(hx - oracle.psf_conv(p, x)) / np.linalg.norm(hx)

    assert err(obs.dl * 8, oracle.NO_DIVIDE_BY_N, coplanar=True) < 1e-12
    e = [err(obs.dl * s) for s in (1, 4, 16)]
    assert e[0] < e[1] < e[2]
    assert e[0] < 1e-3 and e[2] > 1e-2


# ------------------------------------------------------------------ whole solve
def _clean_case(seed, noise):
    obs = synth.tiny_observation(nx=16, ny=16)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    xt = synth.sparse_random_image(rng, 1, 16, 16, 0.2)
    V = oracle.degrid(*a, xt, obs.dl, obs.dm)
    if noise:
        V = V + synth.complex_noise(rng, (obs.nrow, obs.nchan), noise)
    return obs, a, w, xt, V


def test_clean_stops_at_truth():
    """Started at the true image with noiseless data and lam = 0, the first step is a
    fixed point (the exact residual of Eq. 3 vanishes), so the stopping rule ends the
    solve after one step; the count is that step plus the dirty image and PSF."""
    obs, a, w, xt, V = _clean_case(43, 0.0)
    prm = oracle.Params(gamma=1.0, sigma=1e-2, lam=0.0, cg_iters=20, pd_iters=50)
    r = oracle.clean(*a, V, w, 16, 16, obs.dl, obs.dm, 1, prm, max_outer=5, tol=1e-8, x0=xt)
    assert r["n_outer"] == 1 and r["n_hessian"] == 2
    assert np.abs(r["x"] - xt).max() < 1e-9
    assert r["history"][0, 1] < 1e-9


def test_clean_driver_counts_and_composition():
    """tol <= 0 runs max_outer steps, each the step of Eqs. 6-7 applied to the
    previous iterate; with the approximate gradient no step counts as a Hessian."""
    obs, a, w, xt, V = _clean_case(44, 1e-3)
    prm = oracle.Params(gamma=1.0, sigma=1e-2, lam=1e-3, cg_iters=8, pd_iters=10)
    r = oracle.clean(*a, V, w, 16, 16, obs.dl, obs.dm, 1, prm, max_outer=3, tol=0.0)
    assert r["n_outer"] == 3 and r["n_hessian"] == 4
    assert r["history"].shape == (3, 3)
    x = np.zeros((1, 16, 16)); v = np.zeros((1, 1, 16, 16))
    for k in range(3):
        x, v, st = oracle.step(*a, w, r["dirty"], r["psf"], r["wsum"], x, v, obs.dl, obs.dm, prm)
        assert np.array_equal(st, r["history"][k])
    assert np.array_equal(x, r["x"])
    assert r["history"][-1, 0] < r["history"][0, 0]
    prm.approx_gradient = True
    ra = oracle.clean(*a, V, w, 16, 16, obs.dl, obs.dm, 1, prm, max_outer=2, tol=0.0)
    assert ra["n_outer"] == 2 and ra["n_hessian"] == 1


# ------------------------------------------------------------------ facets (image centre away from the phase centre)
def _facets(nx, ny, fx, fy, dl, dm):
    """(i0, j0, l0, m0) of the fx x fy facets that tile an nx x ny image centred on the phase centre."""
    out = []
    for i0 in range(0, nx, fx):
        for j0 in range(0, ny, fy):
            out.append((i0, j0, (i0 + fx // 2 - nx // 2) * dl, (j0 + fy // 2 - ny // 2) * dm))
    return out


def test_facets_sum_to_the_full_image():
    """R of an image equals the sum of R over facets that tile it, each facet an image of
    its own centred at its (l0, m0); R^dagger of a facet is the full image's R^dagger on
    the facet's pixels.  Both follow from Eq. 1 being a sum over pixels at absolute l, m."""
    obs = synth.tiny_observation(nx=32, ny=24)
    rng = np.random.default_rng(51)
    a = (obs.uvw * 8.0, obs.freq, obs.band_of_chan)
    dl, dm = obs.dl * 3, obs.dm * 3          # a wide field: the w term matters
    x = rng.uniform(0, 1, (1, 32, 24))
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    v_full = oracle.degrid(*a, x, dl, dm)
    i_full = oracle.grid(*a, y, None, 32, 24, dl, dm, 1)
    v_sum = np.zeros_like(v_full)
    for i0, j0, l0, m0 in _facets(32, 24, 16, 12, dl, dm):
        xf = x[:, i0:i0 + 16, j0:j0 + 12]
        v_sum += oracle.degrid(*a, xf, dl, dm, l0=l0, m0=m0)
        i_f = oracle.grid(*a, y, None, 16, 12, dl, dm, 1, l0=l0, m0=m0)
        assert np.abs(i_f - i_full[:, i0:i0 + 16, j0:j0 + 12]).max() < 1e-10 * np.abs(i_full).max()
    assert np.abs(v_sum - v_full).max() < 1e-10 * np.abs(v_full).max()


def test_facet_offset_is_a_shift_when_coplanar():
    """Without the w term and 1/n the offset is the shift theorem:
    R_(l0,m0) x = exp(-2 pi i (u l0 + v m0)) R_(0,0) x."""
    obs = synth.tiny_observation(nx=16, ny=16)
    rng = np.random.default_rng(52)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    x = rng.uniform(0, 1, (1, 16, 16))
    f = oracle.NO_WTERM | oracle.NO_DIVIDE_BY_N
    l0, m0 = 7.5 * obs.dl, -3.25 * obs.dm
    v0 = oracle.degrid(*a, x, obs.dl, obs.dm, flags=f)
    v1 = oracle.degrid(*a, x, obs.dl, obs.dm, flags=f, l0=l0, m0=m0)
    s = obs.freq[None, :] / synth.C_LIGHT
    ph = np.exp(-2j * np.pi * (obs.uvw[:, 0:1] * s * l0 + obs.uvw[:, 1:2] * s * m0))
    assert np.abs(v1 - ph * v0).max() < 1e-12 * np.abs(v0).max()
