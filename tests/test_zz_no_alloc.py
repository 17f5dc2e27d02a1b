"""The allocation-free weight-sum entry point (pfb_wsum_static), called through
the C ABI: its per-band sums must equal those of the context-based path
(pfb_dirty's wsum_out) on two calls in a row.  It exists for callers that may
not allocate device memory when they need the sums (an engine owning the whole
HBM pool, or a stream where an allocation could synchronise the device)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2101_08072_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [32, 64])
def test_wsum_static_matches_context_path(prec):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context, Geometry, _lib
    lib = _lib.load()
    obs = synth.tiny_observation(nx=32, ny=32, nchan=6, nband=3)
    obs.band_of_chan = np.array([0, 0, 1, 2, 2, 2], dtype=np.int32)
    rng = np.random.default_rng(41)
    dt = np.float32 if prec == 32 else np.float64
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan)).astype(dt)
    vis = synth.random_vis(rng, (obs.nrow, obs.nchan)).astype(np.complex64 if prec == 32 else np.complex128)
    dev = torch.device("cuda", 0)
    uvw = torch.from_numpy(obs.uvw).to(dev)
    freq = torch.from_numpy(obs.freq).to(dev)
    band = torch.from_numpy(obs.band_of_chan).to(dev)
    wt = torch.from_numpy(w).to(dev)
    ctx = Context(0)
    g = Geometry(nx=32, ny=32, dl=obs.dl, dm=obs.dm, nband=3, epsilon=1e-5 if prec == 32 else 1e-10)
    _, ref = ctx.pfb_dirty(g, uvw, freq, band, torch.from_numpy(vis).to(dev), wt)
    ctx.close()
    out = torch.full((3,), -1.0, dtype=torch.float64, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for _ in range(2):      # the shared accumulators must be cleared by every call
        rc = lib.pfb_wsum_static(0, 0 if prec == 32 else 1, obs.nrow, obs.nchan, 3,
                                 ctypes.c_void_p(band.data_ptr()), ctypes.c_void_p(wt.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.pfb_last_error(None)
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=0.0), (got, ref)
    rc = lib.pfb_wsum_static(0, 0, obs.nrow, obs.nchan, 33, ctypes.c_void_p(band.data_ptr()),
                             ctypes.c_void_p(wt.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == -1 and b"maximum" in lib.pfb_last_error(None)
