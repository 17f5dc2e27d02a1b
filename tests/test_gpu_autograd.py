"""Autograd through R (differentiation workload: 2048^2 image, 1 band, 16 channels
over 0.856-1.712 GHz, MeerKAT-like rows, x a non-negative sparse image at 1% density):
the backward pass (the gridding adjoint) against central finite differences on
32 random pixels and against the FP64 oracle gradient R^dagger Sigma^-1 (R x - V)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_08072_gb300 import synth
from gpu_common import rel_l2

pytestmark = pytest.mark.gpu


def _setup(nrow_keep):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context, Geometry
    obs = synth.meerkat_like_observation(nchan=16, nband=1, nx=2048, ny=2048)
    obs = synth.subset_rows(obs, np.arange(nrow_keep))
    rng = np.random.default_rng(61)
    x = synth.sparse_random_image(rng, 1, 2048, 2048, 0.01)
    dev = torch.device("cuda", 0)
    d = dict(obs=obs, dev=dev, ctx=Context(0), rng=rng,
             g=Geometry(nx=2048, ny=2048, dl=obs.dl, dm=obs.dm, nband=1, epsilon=1e-5),
             uvw=torch.from_numpy(obs.uvw).to(dev), freq=torch.from_numpy(obs.freq).to(dev),
             band=torch.from_numpy(obs.band_of_chan.astype(np.int32)).to(dev), x=x)
    return d


def test_backward_matches_central_differences():
    from paper_2101_08072_gb300.autograd import data_fidelity
    d = _setup(200_000)
    obs, dev = d["obs"], d["dev"]
    rng = d["rng"]
    w = torch.from_numpy(rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan)).astype(np.float32)).to(dev)
    vis = torch.from_numpy(synth.random_vis(rng, (obs.nrow, obs.nchan)).astype(np.complex64)).to(dev)
    x = torch.from_numpy(d["x"].astype(np.float32)).to(dev).requires_grad_(True)
    args = (vis, w, d["g"], d["uvw"], d["freq"], d["band"], d["ctx"])
    f = data_fidelity(x, *args)
    f.backward()
    g = x.grad.detach().double().cpu().numpy().reshape(-1)
    pix = rng.choice(2048 * 2048, 32, replace=False)
    # f is quadratic, so any step is exact up to rounding; a large one keeps FP32 noise small
    h = 0.25 * float(x.detach().max())
    fd = []
    with torch.no_grad():
        for p in pix:
            xp = x.detach().clone(); xp.view(-1)[p] += h
            xm = x.detach().clone(); xm.view(-1)[p] -= h
            fd.append(float(data_fidelity(xp, *args) - data_fidelity(xm, *args)) / (2 * h))
    fd = np.array(fd)
    assert rel_l2(g[pix], fd) <= 2e-3
    d["ctx"].close()


def test_gradient_matches_oracle():
    from paper_2101_08072_gb300.autograd import data_fidelity
    d = _setup(1500)
    obs, dev, rng = d["obs"], d["dev"], d["rng"]
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan))
    V = synth.random_vis(rng, (obs.nrow, obs.nchan))
    x = torch.from_numpy(d["x"].astype(np.float32)).to(dev).requires_grad_(True)
    f = data_fidelity(x, torch.from_numpy(V.astype(np.complex64)).to(dev),
                      torch.from_numpy(w.astype(np.float32)).to(dev), d["g"], d["uvw"], d["freq"], d["band"], d["ctx"])
    f.backward()
    pix = np.sort(rng.choice(2048 * 2048, 64, replace=False))
    x64 = x.detach().double().cpu().numpy()
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    rx = oracle.degrid(*a, x64, obs.dl, obs.dm)
    Vr = V.astype(np.complex64).astype(np.complex128)
    wr = w.astype(np.float32).astype(np.float64)
    ref = oracle.grid(*a, rx - Vr, wr, 2048, 2048, obs.dl, obs.dm, 1, pix=pix)
    got = x.grad.double().cpu().numpy().reshape(-1)[pix]
    assert rel_l2(got, ref) <= 3e-5
    d["ctx"].close()
