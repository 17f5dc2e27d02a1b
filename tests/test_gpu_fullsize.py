"""Parity at the benchmark's full size and launch configuration (the MeerKAT-like
workload: 907,200 rows x 256 channels, 4 bands, 4096^2 pixels, FP32 at
epsilon = 3e-5): sampled outputs computed one by one by the FP64 oracle, and
properties that hold at any size."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_08072_gb300 import synth
from gpu_common import rel_l2

pytestmark = pytest.mark.gpu

EPS = 3e-5
TOL = 3e-5


@pytest.fixture(scope="module")
def big():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context, Geometry
    obs = synth.meerkat_like_observation()
    rng = np.random.default_rng(2)
    bf = synth.band_centre_freqs(obs.freq, obs.band_of_chan, obs.nband)
    x = synth.point_source_image(rng, obs.nband, obs.nx, obs.ny, 1000, flux="pareto", fmin=1e-3, fmax=1.0,
                                 spectral=True, band_freqs=bf)
    dev = torch.device("cuda", 0)
    d = dict(obs=obs, x=x, dev=dev, ctx=Context(0),
             g=Geometry(nx=obs.nx, ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=EPS),
             uvw=torch.from_numpy(obs.uvw).to(dev), freq=torch.from_numpy(obs.freq).to(dev),
             band=torch.from_numpy(obs.band_of_chan.astype(np.int32)).to(dev),
             xt=torch.from_numpy(x.astype(np.float32)).to(dev))
    yield d
    d["ctx"].close()


def test_degrid_sampled_rows(big):
    obs = big["obs"]
    v = big["ctx"].pfb_degrid(big["g"], big["uvw"], big["freq"], big["band"], big["xt"])
    rows = np.sort(np.random.default_rng(11).choice(obs.nrow, 24, replace=False))
    ref = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, big["xt"].cpu().numpy().astype(np.float64),
                        obs.dl, obs.dm, rows=rows)
    got = v[torch.from_numpy(rows).to(big["dev"])].cpu().numpy()
    assert rel_l2(got, ref) <= TOL


def test_grid_sampled_pixels(big):
    obs = big["obs"]
    rng = np.random.default_rng(12)
    y = synth.random_vis(rng, (obs.nrow, obs.nchan)).astype(np.complex64)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan)).astype(np.float32)
    dev = big["dev"]
    img = big["ctx"].pfb_grid(big["g"], big["uvw"], big["freq"], big["band"], torch.from_numpy(y).to(dev),
                              torch.from_numpy(w).to(dev))
    npx = obs.nband * obs.nx * obs.ny
    pix = np.sort(np.random.default_rng(13).choice(npx, 256, replace=False))
    ref = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y.astype(np.complex128), w.astype(np.float64),
                      obs.nx, obs.ny, obs.dl, obs.dm, obs.nband, pix=pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev)].cpu().numpy()
    assert rel_l2(got, ref) <= TOL


def test_hessian_properties_full_size(big):
    """H x = R^dagger (W . R x) as composed calls, and <H x, z> = <x, H z>."""
    obs, ctx, g, dev = big["obs"], big["ctx"], big["g"], big["dev"]
    gen = torch.Generator(device=dev)
    gen.manual_seed(14)
    w = torch.empty((obs.nrow, obs.nchan), dtype=torch.float32, device=dev).uniform_(0.5, 1.5, generator=gen)
    a = (g, big["uvw"], big["freq"], big["band"])
    hx = ctx.pfb_hessian(*a, big["xt"], w)
    v = ctx.pfb_degrid(*a, big["xt"])
    hx2 = ctx.pfb_grid(*a, v, w)
    assert rel_l2(hx.cpu().numpy(), hx2.cpu().numpy()) <= 1e-6
    z = torch.empty_like(big["xt"]).uniform_(-1, 1, generator=gen)
    hz = ctx.pfb_hessian(*a, z, w)
    lhs = float((hx.double() * z.double()).sum())
    rhs = float((big["xt"].double() * hz.double()).sum())
    scale = float(hx.double().norm() * z.double().norm())
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_hessian_row_subset_vs_oracle(big):
    """The Hessian of a row subset at the full image size, at sampled pixels."""
    obs, ctx, g, dev = big["obs"], big["ctx"], big["g"], big["dev"]
    rows = np.sort(np.random.default_rng(15).choice(obs.nrow, 192, replace=False))
    sub = synth.subset_rows(obs, rows)
    w = np.random.default_rng(16).uniform(0.5, 1.5, (sub.nrow, sub.nchan)).astype(np.float32)
    uvw = torch.from_numpy(sub.uvw).to(dev)
    hx = ctx.pfb_hessian(g, uvw, big["freq"], big["band"], big["xt"], torch.from_numpy(w).to(dev))
    x64 = big["xt"].cpu().numpy().astype(np.float64)
    v = oracle.degrid(sub.uvw, sub.freq, sub.band_of_chan, x64, sub.dl, sub.dm)
    npx = obs.nband * obs.nx * obs.ny
    pix = np.sort(np.random.default_rng(17).choice(npx, 64, replace=False))
    ref = oracle.grid(sub.uvw, sub.freq, sub.band_of_chan, v, w.astype(np.float64), obs.nx, obs.ny, obs.dl,
                      obs.dm, obs.nband, pix=pix)
    got = hx.reshape(-1)[torch.from_numpy(pix).to(dev)].cpu().numpy()
    assert rel_l2(got, ref) <= 3 * TOL


def test_fp64_path_full_size_sampled(big):
    """The FP64 path (epsilon = 1e-10) at the full size: R at sampled rows and R^dagger at
    sampled pixels against the oracle, within the FP64 tolerance 1e-9."""
    from paper_2101_08072_gb300 import Geometry
    obs, ctx, dev = big["obs"], big["ctx"], big["dev"]
    g64 = Geometry(nx=obs.nx, ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=1e-10)
    a = (g64, big["uvw"], big["freq"], big["band"])
    x64 = big["xt"].double()
    v = ctx.pfb_degrid(*a, x64)
    rows = np.sort(np.random.default_rng(18).choice(obs.nrow, 16, replace=False))
    ref = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x64.cpu().numpy(), obs.dl, obs.dm, rows=rows)
    got = v[torch.from_numpy(rows).to(dev)].cpu().numpy()
    assert rel_l2(got, ref) <= 1e-9
    del v
    rng = np.random.default_rng(19)
    y = synth.random_vis(rng, (obs.nrow, obs.nchan))
    img = ctx.pfb_grid(*a, torch.from_numpy(y).to(dev))
    npx = obs.nband * obs.nx * obs.ny
    pix = np.sort(np.random.default_rng(20).choice(npx, 64, replace=False))
    ref = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, y, None, obs.nx, obs.ny, obs.dl, obs.dm, obs.nband,
                      pix=pix)
    got = img.reshape(-1)[torch.from_numpy(pix).to(dev)].cpu().numpy()
    assert rel_l2(got, ref) <= 1e-9


def _near_and_random(rng, centres, nband, nx, ny, n_near, n_rand):
    """Flat pixel indices: n_near within 3 pixels of the given (b, i, j) centres, n_rand uniform."""
    out = set()
    while len(out) < n_near:
        b, i, j = centres[rng.integers(len(centres))]
        di, dj = rng.integers(-3, 4, 2)
        out.add(int(b * nx * ny + ((i + di) % nx) * ny + (j + dj) % ny))
    while len(out) < n_near + n_rand:
        out.add(int(rng.integers(nband * nx * ny)))
    return np.array(sorted(out), dtype=np.int64)


def test_psf_sampled_pixels(big):
    """pfb_psf at the full size: the 8192^2 PSF of the 4096^2 image (16384^2 w-planes, whose transforms
    take the full-plane path), against the oracle at pixels around the peak and at random."""
    obs, ctx, dev = big["obs"], big["ctx"], big["dev"]
    rng = np.random.default_rng(21)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan)).astype(np.float32)
    psf, wsum = ctx.pfb_psf(big["g"], big["uvw"], big["freq"], big["band"], torch.from_numpy(w).to(dev))
    n2x, n2y = 2 * obs.nx, 2 * obs.ny
    pix = _near_and_random(rng, [(b, obs.nx, obs.ny) for b in range(obs.nband)], obs.nband, n2x, n2y, 32, 32)
    ones = np.ones((obs.nrow, obs.nchan), dtype=np.complex128)
    ref = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, ones, w.astype(np.float64), n2x, n2y, obs.dl, obs.dm,
                      obs.nband, pix=pix)
    got = psf.reshape(-1)[torch.from_numpy(pix).to(dev)].cpu().numpy()
    assert rel_l2(got, ref) <= TOL
    ws_ref = oracle.wsum(obs.band_of_chan, w.astype(np.float64), obs.nrow, obs.nband)
    assert np.allclose(wsum, ws_ref, rtol=1e-9)
    del psf
    ctx.pfb_plan_reset()


def test_hessian_all_rows_sampled(big):
    """The Hessian on all 907,200 rows (the bench's plan: heavy tiles in chunks that add into zeroed
    cells, light tiles stored whole) at pixels near the sources and at random, for a sparse sky whose
    direct-sum evaluation stays in seconds."""
    obs, ctx, g, dev = big["obs"], big["ctx"], big["g"], big["dev"]
    rng = np.random.default_rng(22)
    x = synth.point_source_image(rng, obs.nband, obs.nx, obs.ny, 16)
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan)).astype(np.float32)
    hx = ctx.pfb_hessian(g, big["uvw"], big["freq"], big["band"], torch.from_numpy(x.astype(np.float32)).to(dev),
                         torch.from_numpy(w).to(dev))
    src = [tuple(int(t) for t in c) for c in np.argwhere(x != 0)]
    pix = _near_and_random(rng, src, obs.nband, obs.nx, obs.ny, 48, 16)
    x32 = x.astype(np.float32).astype(np.float64)
    v = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x32, obs.dl, obs.dm)
    ref = oracle.grid(obs.uvw, obs.freq, obs.band_of_chan, v, w.astype(np.float64), obs.nx, obs.ny, obs.dl,
                      obs.dm, obs.nband, pix=pix)
    got = hx.reshape(-1)[torch.from_numpy(pix).to(dev)].cpu().numpy()
    assert rel_l2(got, ref) <= 2 * TOL
