"""Repeated and interleaved calls on one context.  The w-plane FFT inputs keep their
zero padding (degridding) and their empty tiles (gridding) between calls, cleared
once per plan; these tests check that no call sees data left by another: the same
input gives the same output after other inputs, other plans (the PSF's 2x field)
and other operators ran on the context."""
import numpy as np
import pytest

import oracle
from paper_2101_08072_gb300 import synth
from gpu_common import EPS32, EPS64, TOL32, TOL64, cx_t, dev_obs, geometry, real_t, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_repeated_calls_see_no_stale_data(ctx, prec):
    eps, tol = (EPS32, TOL32) if prec == 32 else (EPS64, TOL64)
    obs = synth.tiny_observation(nx=48, ny=40, nband=2)
    rng = np.random.default_rng(301)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    g = geometry(obs, eps)
    d = dev_obs(obs)
    x1 = synth.point_source_image(rng, 2, 48, 40, 5)
    x2 = synth.point_source_image(rng, 2, 48, 40, 7)
    y1 = synth.random_vis(rng, (obs.nrow, obs.nchan))
    y2 = synth.random_vis(rng, (obs.nrow, obs.nchan))
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    wt = real_t(w, prec)
    v1 = ctx.pfb_degrid(g, *d, real_t(x1, prec)).cpu().numpy()
    i1 = ctx.pfb_grid(g, *d, cx_t(y1, prec), wt).cpu().numpy()
    v2 = ctx.pfb_degrid(g, *d, real_t(x2, prec)).cpu().numpy()
    i2 = ctx.pfb_grid(g, *d, cx_t(y2, prec), wt).cpu().numpy()
    ctx.pfb_psf(g, *d, wt)                          # another plan through the same buffers
    v1b = ctx.pfb_degrid(g, *d, real_t(x1, prec)).cpu().numpy()
    i1b = ctx.pfb_grid(g, *d, cx_t(y1, prec), wt).cpu().numpy()
    assert rel_l2(v2, oracle.degrid(*a, x2, obs.dl, obs.dm)) <= tol
    assert rel_l2(i2, oracle.grid(*a, y2, w, 48, 40, obs.dl, obs.dm, 2)) <= tol
    assert rel_l2(v1, oracle.degrid(*a, x1, obs.dl, obs.dm)) <= tol
    assert rel_l2(i1, oracle.grid(*a, y1, w, 48, 40, obs.dl, obs.dm, 2)) <= tol
    # same input, same output (to the rounding of order-dependent shared-memory sums)
    assert rel_l2(v1b, v1) <= 1e-12
    assert rel_l2(i1b, i1) <= (1e-6 if prec == 32 else 1e-13)


def test_geometry_change_between_calls(ctx):
    """A different image size on the same context after the kept buffers were cleared for another."""
    obs = synth.tiny_observation(nx=32, ny=32, nband=2)
    rng = np.random.default_rng(302)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    x = synth.point_source_image(rng, 2, 32, 32, 4)
    v = ctx.pfb_degrid(geometry(obs, EPS32), *dev_obs(obs), real_t(x, 32)).cpu().numpy()
    assert rel_l2(v, oracle.degrid(*a, x, obs.dl, obs.dm)) <= TOL32
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    im = ctx.pfb_grid(geometry(obs, EPS32), *dev_obs(obs), cx_t(y, 32)).cpu().numpy()
    assert rel_l2(im, oracle.grid(*a, y, None, 32, 32, obs.dl, obs.dm, 2)) <= TOL32
