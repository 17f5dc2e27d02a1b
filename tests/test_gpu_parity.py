"""GPU path (through the C ABI) against the FP64 oracle, element by element on
the same seeded inputs, at sizes the oracle finishes in seconds."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_08072_gb300 import synth
from gpu_common import (EPS32, EPS64, TOL32, TOL64, cx_t, dev_obs, geometry, real_t, rel_l2,
                        wide_observation)

pytestmark = pytest.mark.gpu

PRECS = [(32, EPS32, TOL32), (64, EPS64, TOL64)]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _tiny():
    obs = synth.tiny_observation()
    rng = np.random.default_rng(101)
    x = synth.point_source_image(rng, 1, obs.nx, obs.ny, 5)
    return obs, x, rng


@pytest.mark.parametrize("prec,eps,tol", PRECS)
def test_degrid_tiny(ctx, prec, eps, tol):
    obs, x, _ = _tiny()
    ref = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    v = ctx.pfb_degrid(geometry(obs, eps), *dev_obs(obs), real_t(x, prec)).cpu().numpy()
    assert rel_l2(v, ref) <= tol


@pytest.mark.parametrize("prec,eps,tol", PRECS)
def test_grid_tiny(ctx, prec, eps, tol):
    obs, _, rng = _tiny()
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    ref = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y, w, obs.nx, obs.ny, obs.dl, obs.dm, 1)
    img = ctx.pfb_grid(geometry(obs, eps), *dev_obs(obs), cx_t(y, prec), real_t(w, prec)).cpu().numpy()
    assert rel_l2(img, ref) <= tol


@pytest.mark.parametrize("prec,eps,tol", PRECS)
def test_wide_multiband(ctx, prec, eps, tol):
    """Non-square multi-tile grid, three uneven bands, strong w term."""
    obs = wide_observation()
    rng = np.random.default_rng(102)
    x = synth.point_source_image(rng, obs.nband, obs.nx, obs.ny, 12)
    x += synth.gaussian_blob_image(rng, obs.nband, obs.nx, obs.ny, 2, fwhm_px=(3, 8))
    ref = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    v = ctx.pfb_degrid(geometry(obs, eps), *dev_obs(obs), real_t(x, prec)).cpu().numpy()
    assert rel_l2(v, ref) <= tol
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    ref = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y, w, obs.nx, obs.ny, obs.dl, obs.dm, obs.nband)
    img = ctx.pfb_grid(geometry(obs, eps), *dev_obs(obs), cx_t(y, prec), real_t(w, prec)).cpu().numpy()
    for b in range(obs.nband):
        assert rel_l2(img[b], ref[b]) <= tol, b


def test_item_records_off_matches(ctx):
    """PFB_NO_ITEM_RECORDS (geometry recomputed from uvw in the kernels) gives the
    oracle's result and agrees with the default plan that streams stored item records."""
    from paper_2101_08072_gb300._lib import PFB_NO_ITEM_RECORDS
    obs = wide_observation()
    rng = np.random.default_rng(103)
    x = synth.point_source_image(rng, obs.nband, obs.nx, obs.ny, 12)
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    g_on = geometry(obs, EPS32)
    g_off = geometry(obs, EPS32, flags=PFB_NO_ITEM_RECORDS)
    d = dev_obs(obs)
    ref_v = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    ref_i = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y, w, obs.nx, obs.ny, obs.dl, obs.dm, obs.nband)
    out = {}
    for name, g in (("on", g_on), ("off", g_off)):
        v = ctx.pfb_degrid(g, *d, real_t(x, 32)).cpu().numpy()
        img = ctx.pfb_grid(g, *d, cx_t(y, 32), real_t(w, 32)).cpu().numpy()
        assert rel_l2(v, ref_v) <= TOL32, name
        for b in range(obs.nband):
            assert rel_l2(img[b], ref_i[b]) <= TOL32, (name, b)
        out[name] = (v, img)
    assert rel_l2(out["off"][0], out["on"][0]) <= 1e-6
    assert rel_l2(out["off"][1], out["on"][1]) <= 1e-6


@pytest.mark.parametrize("prec,eps,tol", PRECS)
def test_dirty_psf_hessian(ctx, prec, eps, tol):
    obs = synth.tiny_observation(nx=32, ny=32)
    rng = np.random.default_rng(103)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    x = synth.point_source_image(rng, 1, 32, 32, 4)
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    V = oracle.degrid(*a, x, obs.dl, obs.dm) + synth.complex_noise(rng, (obs.nrow, obs.nchan))
    d_ref, ws_ref = oracle.dirty(*a, V, w, 32, 32, obs.dl, obs.dm, 1)
    p_ref, _ = oracle.psf(*a, w, 32, 32, obs.dl, obs.dm, 1)
    h_ref = oracle.hessian(*a, w, x, obs.dl, obs.dm)
    g = geometry(obs, eps)
    dv = dev_obs(obs)
    d, ws = ctx.pfb_dirty(g, *dv, cx_t(V, prec), real_t(w, prec))
    p, ws2 = ctx.pfb_psf(g, *dv, real_t(w, prec))
    h = ctx.pfb_hessian(g, *dv, real_t(x, prec), real_t(w, prec))
    assert rel_l2(d.cpu().numpy(), d_ref) <= tol
    assert rel_l2(p.cpu().numpy(), p_ref) <= tol
    assert rel_l2(h.cpu().numpy(), h_ref) <= tol
    assert np.allclose(ws, ws_ref, rtol=1e-6 if prec == 32 else 1e-12)
    assert np.allclose(ws2, ws_ref, rtol=1e-6 if prec == 32 else 1e-12)


@pytest.mark.parametrize("prec", [32, 64])
def test_adjoint_pair(ctx, prec):
    """The GPU degrid and grid are mutual adjoints up to rounding."""
    obs = wide_observation(seed=33)
    rng = np.random.default_rng(104)
    x = rng.normal(size=(obs.nband, obs.nx, obs.ny))
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    g = geometry(obs, EPS32 if prec == 32 else EPS64)
    dv = dev_obs(obs)
    rx = ctx.pfb_degrid(g, *dv, real_t(x, prec)).cpu().numpy().astype(np.complex128)
    ry = ctx.pfb_grid(g, *dv, cx_t(y, prec)).cpu().numpy().astype(np.float64)
    xr = real_t(x, prec).cpu().numpy().astype(np.float64)
    yr = cx_t(y, prec).cpu().numpy().astype(np.complex128)
    lhs = float(np.real(np.vdot(rx, yr)))
    rhs = float(np.sum(xr * ry))
    scale = np.linalg.norm(rx) * np.linalg.norm(yr)
    assert abs(lhs - rhs) <= (2e-6 if prec == 32 else 1e-12) * scale


@pytest.mark.parametrize("prec,eps,tol", PRECS)
def test_flags_and_phase_centre(ctx, prec, eps, tol):
    obs, _, rng = _tiny()
    x = np.zeros((1, obs.nx, obs.ny)); x[0, obs.nx // 2, obs.ny // 2] = 1.0
    v = ctx.pfb_degrid(geometry(obs, eps), *dev_obs(obs), real_t(x, prec)).cpu().numpy()
    assert np.abs(v - 1.0).max() <= 3 * tol
    x = synth.point_source_image(rng, 1, obs.nx, obs.ny, 3)
    for flags in (oracle.NO_WTERM, oracle.NO_DIVIDE_BY_N, oracle.NO_WTERM | oracle.NO_DIVIDE_BY_N):
        ref = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm, flags=flags)
        v = ctx.pfb_degrid(geometry(obs, eps, flags), *dev_obs(obs), real_t(x, prec)).cpu().numpy()
        assert rel_l2(v, ref) <= tol, flags


@pytest.mark.parametrize("prec,eps,tol", PRECS)
def test_edge_single_visibility_and_negative_w(ctx, prec, eps, tol):
    obs, x, _ = _tiny()
    one = synth.Observation(uvw=np.array([[123.0, -45.0, -67.0]]), freq=np.array([1.05e9]),
                            band_of_chan=np.array([0], dtype=np.int32), nx=obs.nx, ny=obs.ny, dl=obs.dl,
                            dm=obs.dm, nband=1)
    ref = oracle.degrid(one.uvw, one.freq, one.band_of_chan, x, one.dl, one.dm)
    v = ctx.pfb_degrid(geometry(one, eps), *dev_obs(one), real_t(x, prec)).cpu().numpy()
    assert rel_l2(v, ref) <= tol
    neg = synth.Observation(uvw=-np.abs(obs.uvw), freq=obs.freq, band_of_chan=obs.band_of_chan, nx=obs.nx,
                            ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=1)
    ref = oracle.degrid(neg.uvw, neg.freq, neg.band_of_chan, x, neg.dl, neg.dm)
    v = ctx.pfb_degrid(geometry(neg, eps), *dev_obs(neg), real_t(x, prec)).cpu().numpy()
    assert rel_l2(v, ref) <= tol


@pytest.mark.parametrize("prec", [32, 64])
def test_empty_band_and_zero_weights(ctx, prec):
    obs = synth.tiny_observation(nx=32, ny=32, nchan=4, nband=3)
    obs.band_of_chan = np.array([0, 0, 2, 2], dtype=np.int32)    # band 1 has no channel
    rng = np.random.default_rng(105)
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    w[:, 1] = 0.0
    eps, tol = (EPS32, TOL32) if prec == 32 else (EPS64, TOL64)
    ref = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y, w, 32, 32, obs.dl, obs.dm, 3)
    img = ctx.pfb_grid(geometry(obs, eps), *dev_obs(obs), cx_t(y, prec), real_t(w, prec)).cpu().numpy()
    assert np.abs(img[1]).max() == 0.0
    assert rel_l2(img[0], ref[0]) <= tol and rel_l2(img[2], ref[2]) <= tol


@pytest.mark.parametrize("prec", [32, 64])
def test_psf_conv(ctx, prec):
    rng = np.random.default_rng(106)
    psf = rng.normal(size=(2, 48, 40))
    x = rng.normal(size=(2, 24, 20))
    ref = oracle.psf_conv_direct(psf, x)
    from paper_2101_08072_gb300 import Geometry
    g = Geometry(nx=24, ny=20, dl=1e-5, dm=1e-5, nband=2)
    y = ctx.pfb_psf_conv(g, real_t(psf, prec), real_t(x, prec)).cpu().numpy()
    assert rel_l2(y, ref) <= (1e-5 if prec == 32 else 1e-12)


@pytest.mark.parametrize("prec,mask,nlevel", [(32, 1, 2), (64, 1, 2), (32, 0b1111111, 2), (64, 0b1111111, 2),
                                              (32, 0b1111111, 3), (64, 0b1111111, 3), (64, 0b1111111, 4)])
def test_step_fixed_iterations(ctx, prec, mask, nlevel):
    """One pfb step against the oracle's step at identical iteration counts, with the
    Dirac basis alone and with the full dictionary of Eq. 9 (Dirac + db1..db6), at two to
    four wavelet levels on two bands (the coarse bands of the intermediate levels of every
    band go through scratch between levels)."""
    from paper_2101_08072_gb300 import StepParams
    obs = synth.tiny_observation(nx=32, ny=32, nband=2)
    rng = np.random.default_rng(107)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    xt = synth.point_source_image(rng, 2, 32, 32, 4)
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    V = oracle.degrid(*a, xt, obs.dl, obs.dm) + synth.complex_noise(rng, (obs.nrow, obs.nchan), 1e-4)
    d, ws = oracle.dirty(*a, V, w, 32, 32, obs.dl, obs.dm, 2)
    p, _ = oracle.psf(*a, w, 32, 32, obs.dl, obs.dm, 2)
    x0 = 0.5 * xt
    nbasis = bin(mask).count("1")
    v0 = np.zeros((nbasis, 2, 32, 32))
    prm = oracle.Params(gamma=1.0, sigma=1e-2, lam=1e-3, cg_iters=10, pd_iters=20, nlevel=nlevel, basis_mask=mask)
    x1, v1, st = oracle.step(*a, w, d, p, ws, x0, v0, obs.dl, obs.dm, prm)
    eps = EPS32 if prec == 32 else EPS64
    g = geometry(obs, eps)
    xg, vg = real_t(x0, prec), real_t(v0, prec)
    nh, stg = ctx.pfb_step(g, StepParams(gamma=1.0, sigma=1e-2, lam=1e-3, cg_iters=10, pd_iters=20, nlevel=nlevel,
                                         basis_mask=mask), *dev_obs(obs),
                           real_t(w, prec), real_t(d, prec), real_t(p, prec), ws, xg, vg)
    tol = 1e-4 if prec == 32 else 1e-8
    assert nh == 1
    assert rel_l2(xg.cpu().numpy(), x1) <= tol
    assert rel_l2(vg.cpu().numpy(), v1) <= tol
    assert stg[0] == pytest.approx(st[0], rel=tol, abs=tol * abs(st[0]) + 1e-12)
    assert stg[1] == pytest.approx(st[1], rel=10 * tol)


def test_errors(ctx):
    from paper_2101_08072_gb300 import PfbError, Geometry
    obs, x, _ = _tiny()
    with pytest.raises(PfbError) as e:
        ctx.pfb_degrid(geometry(obs, 1e-8), *dev_obs(obs), real_t(x, 32))
    assert e.value.code == -4
    g = Geometry(nx=63, ny=64, dl=obs.dl, dm=obs.dm)
    with pytest.raises(PfbError) as e:
        ctx.pfb_degrid(g, *dev_obs(obs), real_t(np.zeros((1, 63, 64)), 32))
    assert e.value.code == -1
    bad = synth.Observation(uvw=obs.uvw, freq=obs.freq, band_of_chan=np.array([0, 0, 5, 0], dtype=np.int32),
                            nx=obs.nx, ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=1)
    with pytest.raises(PfbError) as e:
        ctx.pfb_degrid(geometry(bad, 1e-5), *dev_obs(bad), real_t(x, 32))
    assert e.value.code == -1
