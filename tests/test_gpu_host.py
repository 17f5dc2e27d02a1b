"""pfb_hessian_host: the Hessian from host buffers with the copies overlapped, against the FP64
oracle and against pfb_hessian on device buffers; a new set of host arrays rebuilds the plan."""
import numpy as np
import pytest
import torch

import oracle
from paper_2101_08072_gb300 import synth
from gpu_common import EPS32, EPS64, TOL32, TOL64, dev_obs, geometry, real_t, rel_l2, wide_observation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _host(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).pin_memory()


def _host_obs(obs):
    return (_host(obs.uvw, np.float64), _host(obs.freq, np.float64), _host(obs.band_of_chan, np.int32))


@pytest.mark.parametrize("prec,eps,tol", [(32, EPS32, TOL32), (64, EPS64, TOL64)])
@pytest.mark.parametrize("weighted", [True, False])
def test_hessian_host_matches_oracle(ctx, prec, eps, tol, weighted):
    obs = wide_observation()
    rng = np.random.default_rng(401)
    a = (obs.uvw, obs.freq, obs.band_of_chan)
    x = synth.point_source_image(rng, obs.nband, obs.nx, obs.ny, 10)
    w = synth.uniform_weights(rng, (obs.nrow, obs.nchan)) if weighted else None
    ref = oracle.hessian(*a, w, x, obs.dl, obs.dm)
    rdt = np.float64 if prec == 64 else np.float32
    hw = _host(w, rdt) if weighted else None
    y = ctx.pfb_hessian_host(geometry(obs, eps), *_host_obs(obs), _host(x, rdt), hw)
    torch.cuda.current_stream().synchronize()
    assert y.device.type == "cpu"
    assert rel_l2(y.numpy(), ref) <= tol
    # the device-buffer entry point on the same inputs
    yd = ctx.pfb_hessian(geometry(obs, eps), *dev_obs(obs), real_t(x, prec),
                         real_t(w, prec) if weighted else None).cpu().numpy()
    assert rel_l2(y.numpy(), yd) <= (1e-6 if prec == 32 else 1e-12)


def test_new_host_arrays_rebuild_the_plan(ctx):
    """Two observations through the host entry point in turn (the same scratch copies on the
    device): each result matches the oracle for its own uvw."""
    rng = np.random.default_rng(402)
    held = []
    for seed in (1, 2, 1):
        obs = synth.tiny_observation(seed=seed, nx=64, ny=64, nband=1)
        a = (obs.uvw, obs.freq, obs.band_of_chan)
        x = synth.point_source_image(rng, 1, 64, 64, 5)
        w = synth.uniform_weights(rng, (obs.nrow, obs.nchan))
        ref = oracle.hessian(*a, w, x, obs.dl, obs.dm)
        ho = _host_obs(obs)
        held.append(ho)
        y = ctx.pfb_hessian_host(geometry(obs, EPS32), *ho, _host(x, np.float32), _host(w, np.float32))
        torch.cuda.current_stream().synchronize()
        assert rel_l2(y.numpy(), ref) <= TOL32, seed
