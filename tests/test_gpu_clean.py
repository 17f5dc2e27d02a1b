"""The whole solve (pfb_clean) and the approximate-gradient step (Eq. 4) through the
C ABI against the FP64 oracle, on the same seeded inputs and iteration counts."""
import functools

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


def _case(seed, noise, nband=2, n=32):
    obs = synth.tiny_observation(nx=n, ny=n, nband=nband)
    rng = np.random.default_rng(seed)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    xt = synth.point_source_image(rng, nband, n, n, 4)
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    V = oracle.degrid(*a, xt, obs.dl, obs.dm)
    if noise:
        V = V + synth.complex_noise(rng, (obs.nrow, obs.nchan), noise)
    return obs, a, xt, w, V


def _params(**kw):
    from paper_2101_08072_gb300 import StepParams
    base = dict(gamma=1.0, sigma=1e-2, lam=1e-3, cg_iters=10, pd_iters=20, nlevel=2, basis_mask=1)
    base.update(kw)
    return StepParams(**base), oracle.Params(**base)


@pytest.mark.parametrize("prec", [32, 64])
def test_approx_gradient_step(ctx, prec):
    """A step with PFB_STEP_APPROX_GRADIENT (IR = I^d - I^psf * x_k) against the oracle's."""
    obs, a, xt, w, V = _case(201, 1e-4)
    d, ws = oracle.dirty(*a, V, w, 32, 32, obs.dl, obs.dm, 2)
    p, _ = oracle.psf(*a, w, 32, 32, obs.dl, obs.dm, 2)
    x0 = 0.5 * xt
    v0 = np.zeros((1, 2, 32, 32))
    gp, op = _params(approx_gradient=True)
    x1, v1, st = oracle.step(*a, w, d, p, ws, x0, v0, obs.dl, obs.dm, op)
    g = geometry(obs, EPS32 if prec == 32 else EPS64)
    xg, vg = real_t(x0, prec), real_t(v0, prec)
    nh, stg = ctx.pfb_step(g, gp, *dev_obs(obs), real_t(w, prec), real_t(d, prec), real_t(p, prec), ws, xg, vg)
    tol = 1e-4 if prec == 32 else 1e-8
    assert nh == 0
    assert rel_l2(xg.cpu().numpy(), x1) <= tol
    assert rel_l2(vg.cpu().numpy(), v1) <= tol
    assert stg[0] == pytest.approx(st[0], rel=tol)


@functools.lru_cache(maxsize=None)
def _large_case(mask):
    nx, ny, nb = 1288, 1000, 2
    obs = synth.tiny_observation(nx=32, ny=32, nband=nb)
    rng = np.random.default_rng(203)
    ws = np.array([1.0, 1.25])
    ii = np.arange(2 * nx)[:, None] - nx
    jj = np.arange(2 * ny)[None, :] - ny
    beam = np.exp(-(ii * ii + jj * jj) / (2.0 * 2.5 ** 2))
    p = ws[:, None, None] * beam[None]
    xt = synth.point_source_image(rng, nb, nx, ny, 60)
    d = oracle.psf_conv(p, xt) + 1e-3 * rng.normal(size=(nb, nx, ny))
    x0 = 0.5 * xt
    v0 = np.zeros((bin(mask).count("1"), nb, nx, ny))
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
    _, op = _params(approx_gradient=True, cg_iters=4, pd_iters=4, basis_mask=mask)
    ref = oracle.step(obs.uvw, obs.freq, obs.band_of_chan, w, d, p, ws, x0, v0, obs.dl, obs.dm, op)
    return obs, w, ws, p, d, x0, v0, ref


@pytest.mark.parametrize("prec,mask", [(32, 1), (32, 0b1111111), (64, 0b1111111)])
def test_approx_gradient_step_large(ctx, prec, mask):
    """The image side of a step (PSF convolution, CG, primal-dual with Dirac + db1..db6) at
    1288 x 1000 pixels: more rows than the image kernels launch CTAs per band, so every
    CTA strides over several rows, and 1000-pixel rows leave a ragged tail of 232 threads.
    The PSF is a Gaussian beam (a positive spectrum, so U is positive definite); the
    dirty image its convolution with point sources plus noise."""
    nx, ny, nb = 1288, 1000, 2
    obs, w, ws, p, d, x0, v0, (x1, v1, st) = _large_case(mask)
    gp, _ = _params(approx_gradient=True, cg_iters=4, pd_iters=4, basis_mask=mask)
    from paper_2101_08072_gb300 import Geometry
    g = Geometry(nx=nx, ny=ny, dl=obs.dl, dm=obs.dm, nband=nb, epsilon=EPS32 if prec == 32 else EPS64)
    xg, vg = real_t(x0, prec), real_t(v0, prec)
    nh, stg = ctx.pfb_step(g, gp, *dev_obs(obs), real_t(w, prec), real_t(d, prec), real_t(p, prec), ws, xg, vg)
    tol = 1e-4 if prec == 32 else 1e-8
    assert nh == 0
    assert rel_l2(xg.cpu().numpy(), x1) <= tol
    assert rel_l2(vg.cpu().numpy(), v1) <= tol
    assert stg[0] == pytest.approx(st[0], rel=tol)
    assert stg[1] == pytest.approx(st[1], rel=10 * tol)


@pytest.mark.parametrize("prec,mask", [(32, 1), (64, 1), (64, 0b101)])
def test_clean_fixed_iterations(ctx, prec, mask):
    """pfb_clean with tol = 0 (max_outer steps) against oracle.clean: PSF, dirty image,
    weight sums, final iterate, dual, counts and the per-step statistics."""
    obs, a, xt, w, V = _case(202, 1e-3)
    gp, op = _params(basis_mask=mask)
    ref = oracle.clean(*a, V, w, 32, 32, obs.dl, obs.dm, 2, op, max_outer=3, tol=0.0)
    eps, tol_op = (EPS32, TOL32) if prec == 32 else (EPS64, TOL64)
    g = geometry(obs, eps)
    r = ctx.pfb_clean(g, gp, *dev_obs(obs), cx_t(V, prec), real_t(w, prec), max_outer=3, tol=0.0)
    assert r["n_outer"] == 3 and r["n_hessian"] == 4
    # FP32 weights are the FP64 ones rounded to float32 before they are summed
    assert np.allclose(r["wsum"], ref["wsum"], rtol=1e-12 if prec == 64 else 1e-6)
    assert rel_l2(r["psf"].cpu().numpy(), ref["psf"]) <= tol_op
    assert rel_l2(r["dirty"].cpu().numpy(), ref["dirty"]) <= tol_op
    tol = 1e-4 if prec == 32 else 1e-8
    assert rel_l2(r["x"].cpu().numpy(), ref["x"]) <= tol
    assert rel_l2(r["dual"].cpu().numpy(), ref["dual"]) <= tol
    assert np.allclose(r["history"][:, 0], ref["history"][:, 0], rtol=tol)


@pytest.mark.parametrize("prec", [32, 64])
def test_clean_stops_at_truth(ctx, prec):
    """Noiseless data, lam = 0, started at the true image: the first step is a fixed
    point, so the stopping rule ends the solve after one step (n_hessian = 2)."""
    obs, a, xt, w, V = _case(203, 0.0)
    gp, _ = _params(lam=0.0, cg_iters=20, pd_iters=30)
    g = geometry(obs, EPS32 if prec == 32 else EPS64)
    tol = 1e-3 if prec == 32 else 1e-7
    r = ctx.pfb_clean(g, gp, *dev_obs(obs), cx_t(V, prec), real_t(w, prec), max_outer=5, tol=tol,
                      x=real_t(xt, prec))
    assert r["n_outer"] == 1 and r["n_hessian"] == 2
    assert r["history"][0, 1] <= tol
    assert rel_l2(r["x"].cpu().numpy(), xt) <= (1e-4 if prec == 32 else 1e-8)


def test_clean_equals_its_parts(ctx):
    """pfb_clean is pfb_psf, pfb_dirty and pfb_step in sequence (FP64, 2 steps)."""
    obs, a, xt, w, V = _case(204, 1e-3)
    gp, _ = _params()
    g = geometry(obs, EPS64)
    uvw, freq, band = dev_obs(obs)
    wt, vt = real_t(w, 64), cx_t(V, 64)
    r = ctx.pfb_clean(g, gp, uvw, freq, band, vt, wt, max_outer=2, tol=0.0)
    ctx.pfb_plan_reset()
    psf, ws = ctx.pfb_psf(g, uvw, freq, band, wt)
    ctx.pfb_plan_reset()
    d, _ = ctx.pfb_dirty(g, uvw, freq, band, vt, wt)
    x = real_t(np.zeros((2, 32, 32)), 64)
    v = real_t(np.zeros((1, 2, 32, 32)), 64)
    for k in range(2):
        _, st = ctx.pfb_step(g, gp, uvw, freq, band, wt, d, psf, ws, x, v)
        assert st[0] == pytest.approx(r["history"][k, 0], rel=1e-10)
    assert rel_l2(r["x"].cpu().numpy(), x.cpu().numpy()) <= 1e-10
    assert rel_l2(r["psf"].cpu().numpy(), psf.cpu().numpy()) <= 1e-12


def test_clean_errors(ctx):
    from paper_2101_08072_gb300 import PfbError
    obs, a, xt, w, V = _case(205, 0.0, nband=1, n=16)
    gp, _ = _params()
    g = geometry(obs, EPS64)
    with pytest.raises(PfbError) as e:
        ctx.pfb_clean(g, gp, *dev_obs(obs), cx_t(V, 64), real_t(w, 64), max_outer=-1)
    assert e.value.code == -1
    gp.cg_iters = -2
    with pytest.raises(PfbError) as e:
        ctx.pfb_clean(g, gp, *dev_obs(obs), cx_t(V, 64), real_t(w, 64), max_outer=1)
    assert e.value.code == -1


@pytest.mark.parametrize("prec", [32, 64])
def test_step_bound_against_oracle(ctx, prec):
    """lambda_max(U^-1 H) by power iteration (pfb_step_bound) against the oracle's estimate from the
    same start vector and iteration counts."""
    obs, a, xt, w, V = _case(205, 0.0)
    p, ws = oracle.psf(*a, w, 32, 32, obs.dl, obs.dm, 2)
    z0 = np.random.default_rng(206).uniform(0.5, 1.5, (2, 32, 32))
    gp, op = _params(sigma=0.05, cg_iters=15)
    ref = oracle.step_bound(*a, w, p, ws, obs.dl, obs.dm, op.sigma, 4, op.cg_iters, z0=z0)
    g = geometry(obs, EPS32 if prec == 32 else EPS64)
    got = ctx.pfb_step_bound(g, gp, *dev_obs(obs), real_t(w, prec), real_t(p, prec), ws, iters=4,
                             z0=real_t(z0, prec))
    assert got == pytest.approx(ref, rel=1e-5 if prec == 32 else 1e-10)
    assert ctx.pfb_last_step_bound()[0] == got


@pytest.mark.parametrize("prec", [32, 64])
def test_clean_safe_gamma(ctx, prec):
    """pfb_clean with PFB_STEP_SAFE_GAMMA: the bound from a constant start, gamma capped at 1.9 / bound,
    the bound's Hessians counted; final iterate against the oracle's solve with the same option."""
    obs, a, xt, w, V = _case(207, 1e-4)
    gp, op = _params(gamma=4.0, sigma=0.05, cg_iters=12, pd_iters=10, safe_gamma=True)
    ref = oracle.clean(*a, V, w, 32, 32, obs.dl, obs.dm, 2, op, max_outer=3, tol=0.0)
    g = geometry(obs, EPS32 if prec == 32 else EPS64)
    out = ctx.pfb_clean(g, gp, *dev_obs(obs), cx_t(V, prec), real_t(w, prec), max_outer=3, tol=0.0)
    lm, ga = ctx.pfb_last_step_bound()
    tol = 1e-4 if prec == 32 else 1e-8
    assert lm == pytest.approx(ref["lmax"], rel=tol)
    assert ga == pytest.approx(ref["gamma"], rel=tol) and ga < 4.0
    assert out["n_hessian"] == ref["n_hessian"] == 1 + oracle.BOUND_ITERS + 3
    assert rel_l2(out["x"].cpu().numpy(), ref["x"]) <= tol
