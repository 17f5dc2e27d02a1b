"""Facets through the C ABI: images centred away from the phase centre ((l0, m0) != 0)
against the FP64 oracle, and a faceted image's R (facets accumulated with
PFB_ACCUMULATE) and R^dagger (per facet) against the same operators on the whole image."""
import numpy as np
import pytest

import oracle
from paper_2101_08072_gb300 import synth
from gpu_common import EPS32, EPS64, TOL32, TOL64, cx_t, dev_obs, real_t, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context
    c = Context(0)
    yield c
    c.close()


NX, NY, FX, FY = 64, 48, 32, 24


def _wide():
    """A wide field with a strong w term: the tiny array's baselines stretched, coarse pixels."""
    obs = synth.tiny_observation(nx=NX, ny=NY)
    return synth.Observation(uvw=obs.uvw * 8.0, freq=obs.freq, band_of_chan=obs.band_of_chan, nx=NX, ny=NY,
                             dl=obs.dl * 2.0, dm=obs.dm * 2.0, nband=1)


def _facets(obs):
    out = []
    for i0 in range(0, NX, FX):
        for j0 in range(0, NY, FY):
            out.append((i0, j0, (i0 + FX // 2 - NX // 2) * obs.dl, (j0 + FY // 2 - NY // 2) * obs.dm))
    return out


def _geom(obs, eps, nx, ny, l0=0.0, m0=0.0, flags=0):
    from paper_2101_08072_gb300 import Geometry
    return Geometry(nx=nx, ny=ny, dl=obs.dl, dm=obs.dm, nband=1, epsilon=eps, flags=flags, l0=l0, m0=m0)


@pytest.mark.parametrize("prec", [32, 64])
def test_facet_operators_match_oracle(ctx, prec):
    eps, tol = (EPS32, TOL32) if prec == 32 else (EPS64, TOL64)
    obs = _wide()
    rng = np.random.default_rng(401)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    d = dev_obs(obs)
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    for i0, j0, l0, m0 in _facets(obs)[1:3]:
        x = synth.point_source_image(rng, 1, FX, FY, 6)
        g = _geom(obs, eps, FX, FY, l0, m0)
        v = ctx.pfb_degrid(g, *d, real_t(x, prec)).cpu().numpy()
        assert rel_l2(v, oracle.degrid(*a, x, obs.dl, obs.dm, l0=l0, m0=m0)) <= tol
        im = ctx.pfb_grid(g, *d, cx_t(y, prec), real_t(w, prec)).cpu().numpy()
        assert rel_l2(im, oracle.grid(*a, y, w, FX, FY, obs.dl, obs.dm, 1, l0=l0, m0=m0)) <= tol


@pytest.mark.parametrize("prec", [32, 64])
def test_faceted_image_equals_whole_image(ctx, prec):
    """R x = sum_f R_f x_f (accumulated in one visibility buffer) and R^dagger y on each
    facet's pixels = R_f^dagger y, both against the whole-image GPU operators and the oracle."""
    from paper_2101_08072_gb300 import _lib
    eps, tol = (EPS32, TOL32) if prec == 32 else (EPS64, TOL64)
    obs = _wide()
    rng = np.random.default_rng(402)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    d = dev_obs(obs)
    x = synth.point_source_image(rng, 1, NX, NY, 12)
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    v_full = ctx.pfb_degrid(_geom(obs, eps, NX, NY), *d, real_t(x, prec))
    i_full = ctx.pfb_grid(_geom(obs, eps, NX, NY), *d, cx_t(y, prec)).cpu().numpy()
    v_fac = torch_zeros_like(v_full)
    for i0, j0, l0, m0 in _facets(obs):
        g = _geom(obs, eps, FX, FY, l0, m0, flags=_lib.PFB_ACCUMULATE)
        ctx.pfb_degrid(g, *d, real_t(np.ascontiguousarray(x[:, i0:i0 + FX, j0:j0 + FY]), prec), out=v_fac)
        i_f = ctx.pfb_grid(_geom(obs, eps, FX, FY, l0, m0), *d, cx_t(y, prec)).cpu().numpy()
        assert rel_l2(i_f, i_full[:, i0:i0 + FX, j0:j0 + FY]) <= 2 * tol
    v_ref = oracle.degrid(*a, x, obs.dl, obs.dm)
    assert rel_l2(v_fac.cpu().numpy(), v_ref) <= 2 * tol
    assert rel_l2(v_full.cpu().numpy(), v_ref) <= tol


def test_facet_psf_matches_oracle(ctx):
    obs = _wide()
    rng = np.random.default_rng(403)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    i0, j0, l0, m0 = _facets(obs)[3]
    psf, ws = ctx.pfb_psf(_geom(obs, EPS64, FX, FY, l0, m0), *dev_obs(obs), real_t(w, 64))
    ref, wr = oracle.psf(*a, w, FX, FY, obs.dl, obs.dm, 1, l0=l0, m0=m0)
    assert rel_l2(psf.cpu().numpy(), ref) <= TOL64
    assert np.allclose(ws, wr, rtol=1e-12)


def test_facet_outside_horizon_is_rejected(ctx):
    from paper_2101_08072_gb300 import PfbError
    obs = _wide()
    with pytest.raises(PfbError) as e:
        ctx.pfb_degrid(_geom(obs, EPS32, FX, FY, 0.8, 0.7), *dev_obs(obs), real_t(np.zeros((1, FX, FY)), 32))
    assert e.value.code == -1


def torch_zeros_like(t):
    import torch
    return torch.zeros_like(t)
