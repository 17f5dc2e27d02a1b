"""Pruned plane transforms of the FP32 path (planes of 1024..16384 cells per side, powers of two): only
the image region and the 32 x 32 uv tiles that some visibility touches are transformed, with the pre-
and post-pass folded into the column transforms.  R, R^dagger and the Hessian are checked against the
FP64 oracle and against the full-plane transforms (PFB_NO_PRUNED_FFT) on the same inputs: square and
non-square planes, several bands with an empty one, more than one plane block per band, repeated calls
that reuse the plane buffer, and the 16384-point transforms (one column or row per CTA)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2101_08072_gb300 import synth
from gpu_common import EPS32, TOL32, cx_t, dev_obs, geometry, real_t, rel_l2

pytestmark = pytest.mark.gpu

# The two paths differ only by the rounding of their transforms and phase evaluations.
TOL_PATHS = 2e-6

# (nx, ny, nband): planes 1024 x 1024, 2048 x 1024 and 1024 x 2048
CASES = [(512, 512, 1), (1024, 512, 2), (512, 1024, 1)]


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _no_pruned():
    from paper_2101_08072_gb300 import _lib
    return _lib.PFB_NO_PRUNED_FFT


def _obs(nx, ny, nb, seed=7):
    return synth.tiny_observation(seed=seed, nx=nx, ny=ny, ntime=3, nchan=2 * nb, nband=nb)


def _sky(rng, nb, nx, ny):
    x = synth.point_source_image(rng, nb, nx, ny, 20)
    return x + synth.gaussian_blob_image(rng, nb, nx, ny, 2, fwhm_px=(4, 12))


def _launches(ctx, name):
    n, ms = ctypes.c_int64(0), ctypes.c_double(0)
    ctx.lib.pfb_timing_read(ctx.h, name.encode(), ctypes.byref(n), ctypes.byref(ms), None)
    return n.value


@pytest.mark.parametrize("nx,ny,nb", CASES)
def test_pruned_against_oracle_and_full_planes(ctx, nx, ny, nb):
    obs = _obs(nx, ny, nb)
    rng = np.random.default_rng(311)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    d = dev_obs(obs)
    g = geometry(obs, EPS32)
    gf = geometry(obs, EPS32, flags=_no_pruned())
    ctx.lib.pfb_timing(ctx.h, 1)
    for call in range(2):
        x = _sky(rng, nb, nx, ny)
        ref = oracle.degrid(*a, x, obs.dl, obs.dm)
        v = ctx.pfb_degrid(g, *d, real_t(x, 32)).cpu().numpy()
        vf = ctx.pfb_degrid(gf, *d, real_t(x, 32)).cpu().numpy()
        assert rel_l2(v, ref) <= TOL32, call
        assert rel_l2(v, vf) <= TOL_PATHS, call
        y = synth.random_vis(rng, (obs.nrow, obs.nchan))
        w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
        ref = oracle.grid(*a, y, w, nx, ny, obs.dl, obs.dm, nb)
        img = ctx.pfb_grid(g, *d, cx_t(y, 32), real_t(w, 32)).cpu().numpy()
        imf = ctx.pfb_grid(gf, *d, cx_t(y, 32), real_t(w, 32)).cpu().numpy()
        for b in range(nb):
            assert rel_l2(img[b], ref[b]) <= TOL32, (call, b)
            assert rel_l2(img[b], imf[b]) <= TOL_PATHS, (call, b)
    # the pruned kernels ran (one column pass per band and call in each direction)
    assert _launches(ctx, "col_fwd") == 2 * nb and _launches(ctx, "col_inv") == 2 * nb
    ctx.lib.pfb_timing(ctx.h, 0)


def test_pruned_hessian_and_empty_band(ctx):
    nx = ny = 512
    obs = synth.tiny_observation(seed=9, nx=nx, ny=ny, ntime=3, nchan=4, nband=3)
    obs.band_of_chan = np.array([0, 0, 2, 2], dtype=np.int32)    # band 1 has no channel
    rng = np.random.default_rng(312)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    d = dev_obs(obs)
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    g = geometry(obs, EPS32)
    gf = geometry(obs, EPS32, flags=_no_pruned())
    x = _sky(rng, 3, nx, ny)
    ref = oracle.hessian(*a, w, x, obs.dl, obs.dm)
    hx = ctx.pfb_hessian(g, *d, real_t(x, 32), real_t(w, 32)).cpu().numpy()
    hf = ctx.pfb_hessian(gf, *d, real_t(x, 32), real_t(w, 32)).cpu().numpy()
    assert np.abs(hx[1]).max() == 0.0
    for b in (0, 2):
        assert rel_l2(hx[b], ref[b]) <= TOL32, b
        assert rel_l2(hx[b], hf[b]) <= TOL_PATHS, b


def test_pruned_several_plane_blocks():
    """A budget too small for a whole band's w-stack: the planes go through in blocks, the column pass
    of each later block adds into the image, and the row lists are cut per block."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context
    nx = ny = 512
    obs = _obs(nx, ny, 1, seed=11)
    rng = np.random.default_rng(313)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    d = dev_obs(obs)
    x = _sky(rng, 1, nx, ny)
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    ref = oracle.hessian(*a, w, x, obs.dl, obs.dm)
    g = geometry(obs, EPS32)
    found = False
    for mb in range(96, 512, 8):
        c = Context(0, hbm_budget_bytes=mb << 20)
        try:
            c.lib.pfb_timing(c.h, 1)
            try:
                hx = c.pfb_hessian(g, *d, real_t(x, 32), real_t(w, 32)).cpu().numpy()
            except Exception:
                continue          # budget below one plane block: try a larger one
            blocks = _launches(c, "col_inv")
            if blocks < 2:
                break             # the whole stack fits: larger budgets will not split it
            assert _launches(c, "col_fwd") == blocks
            assert rel_l2(hx, ref) <= TOL32, (mb, blocks)
            found = True
            break
        finally:
            c.close()
    assert found, "no budget split the w-stack into blocks"


# planes of 16384 cells along one axis: the column (8192 x 512 image) or row (512 x 8192 image) transforms
# take single columns / rows per CTA
CASES_16K = [(8192, 512), (512, 8192)]


@pytest.mark.parametrize("nx,ny", CASES_16K)
def test_pruned_16384_point_transforms(ctx, nx, ny):
    obs = _obs(nx, ny, 1, seed=13)
    rng = np.random.default_rng(314)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    d = dev_obs(obs)
    g = geometry(obs, EPS32)
    gf = geometry(obs, EPS32, flags=_no_pruned())
    ctx.lib.pfb_timing(ctx.h, 1)
    x = _sky(rng, 1, nx, ny)
    ref = oracle.degrid(*a, x, obs.dl, obs.dm)
    v = ctx.pfb_degrid(g, *d, real_t(x, 32)).cpu().numpy()
    vf = ctx.pfb_degrid(gf, *d, real_t(x, 32)).cpu().numpy()
    assert rel_l2(v, ref) <= TOL32
    assert rel_l2(v, vf) <= TOL_PATHS
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    img = ctx.pfb_grid(g, *d, cx_t(y, 32), real_t(w, 32)).cpu().numpy()
    imf = ctx.pfb_grid(gf, *d, cx_t(y, 32), real_t(w, 32)).cpu().numpy()
    assert rel_l2(img, imf) <= TOL_PATHS
    pix = np.sort(rng.choice(nx * ny, 1024, replace=False))
    ref = oracle.grid(*a, y, w, nx, ny, obs.dl, obs.dm, 1, pix=pix)
    assert rel_l2(img.reshape(-1)[pix], ref) <= TOL32
    assert _launches(ctx, "col_fwd") == 1 and _launches(ctx, "col_inv") == 1
    ctx.lib.pfb_timing(ctx.h, 0)
