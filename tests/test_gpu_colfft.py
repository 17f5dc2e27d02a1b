"""FP32 planes whose column pass runs in the column-transform kernel (power-of-two Nu from
1024 to 8192; the image columns [0, ny/2) and [Nv - ny/2, Nv), the image rows [0, nx/2) and
[Nu - nx/2, Nu)): R, R^dagger and the Hessian against the FP64 oracle.  Each operator runs
twice with different inputs, so the second call starts from planes and kept-zero buffers
whose columns still hold the first call's transforms."""
import numpy as np
import pytest

import oracle
from paper_2101_08072_gb300 import synth
from gpu_common import EPS32, TOL32, cx_t, dev_obs, geometry, real_t, rel_l2

pytestmark = pytest.mark.gpu

# (nx, ny, nband): planes 1024 x 1024 (radix 16, 16, 4) and 2048 x 1536 (radix 16, 16, 8)
CASES = [(512, 512, 1), (1024, 768, 2)]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _obs(nx, ny, nb):
    return synth.tiny_observation(seed=5, nx=nx, ny=ny, ntime=2, nchan=2 * nb, nband=nb)


@pytest.mark.parametrize("nx,ny,nb", CASES)
def test_degrid_grid(ctx, nx, ny, nb):
    obs = _obs(nx, ny, nb)
    rng = np.random.default_rng(301)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    g = geometry(obs, EPS32)
    for call in range(2):
        x = synth.point_source_image(rng, nb, nx, ny, 20)
        x += synth.gaussian_blob_image(rng, nb, nx, ny, 2, fwhm_px=(4, 12))
        ref = oracle.degrid(*a, x, obs.dl, obs.dm)
        v = ctx.pfb_degrid(g, *dev_obs(obs), real_t(x, 32)).cpu().numpy()
        assert rel_l2(v, ref) <= TOL32, call
        y = synth.random_vis(rng, (obs.nrow, obs.nchan))
        w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
        ref = oracle.grid(*a, y, w, nx, ny, obs.dl, obs.dm, nb)
        img = ctx.pfb_grid(g, *dev_obs(obs), cx_t(y, 32), real_t(w, 32)).cpu().numpy()
        for b in range(nb):
            assert rel_l2(img[b], ref[b]) <= TOL32, (call, b)


@pytest.mark.parametrize("nx,ny,nb", CASES[:1])
def test_hessian(ctx, nx, ny, nb):
    obs = _obs(nx, ny, nb)
    rng = np.random.default_rng(302)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    g = geometry(obs, EPS32)
    for call in range(2):
        x = synth.point_source_image(rng, nb, nx, ny, 20)
        ref = oracle.hessian(*a, w, x, obs.dl, obs.dm)
        hx = ctx.pfb_hessian(g, *dev_obs(obs), real_t(x, 32), real_t(w, 32)).cpu().numpy()
        assert rel_l2(hx, ref) <= TOL32, call
