"""The allocation-free weight-sum entry point (pfb_wsum_static), called through
the C ABI.  It exists for callers that may not allocate device memory when they
need the per-band weight sums: an engine that owns the whole HBM pool, or a
stream where an allocation could synchronise the device.  Its sums must equal
the FP64 oracle's and those of the context-based path (pfb_dirty's wsum_out),
on two calls in a row, with device or host output, with and without weights,
without changing the device's free memory; out-of-range band ids are rejected
as pfb_dirty rejects them."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
from paper_2101_08072_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import _lib as L
    return L.load()


def _call(lib, prec, nrow, nchan, nband, band, wt, out_ptr, dev):
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    return lib.pfb_wsum_static(0, 0 if prec == 32 else 1, nrow, nchan, nband, ctypes.c_void_p(band.data_ptr()),
                               ctypes.c_void_p(wt.data_ptr()) if wt is not None else None,
                               ctypes.c_void_p(out_ptr), stream)


@pytest.mark.parametrize("prec", [32, 64])
def test_wsum_static_matches_oracle_and_context_path(prec):
    from paper_2101_08072_gb300 import Context, Geometry
    lib = _lib()
    obs = synth.tiny_observation(nx=32, ny=32, nchan=6, nband=3)
    obs.band_of_chan = np.array([0, 0, 1, 2, 2, 2], dtype=np.int32)
    rng = np.random.default_rng(41)
    dt = np.float32 if prec == 32 else np.float64
    w = rng.uniform(0.5, 1.5, (obs.nrow, obs.nchan)).astype(dt)
    ref = oracle.wsum(obs.band_of_chan, w.astype(np.float64), obs.nrow, 3)
    ref_unit = oracle.wsum(obs.band_of_chan, None, obs.nrow, 3)
    vis = synth.random_vis(rng, (obs.nrow, obs.nchan)).astype(np.complex64 if prec == 32 else np.complex128)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    uvw = torch.from_numpy(obs.uvw).to(dev)
    freq = torch.from_numpy(obs.freq).to(dev)
    band = torch.from_numpy(obs.band_of_chan).to(dev)
    wt = torch.from_numpy(w).to(dev)
    ctx = Context(0)
    g = Geometry(nx=32, ny=32, dl=obs.dl, dm=obs.dm, nband=3, epsilon=1e-5 if prec == 32 else 1e-10)
    _, ctx_ws = ctx.pfb_dirty(g, uvw, freq, band, torch.from_numpy(vis).to(dev), wt)
    ctx.close()
    assert np.allclose(ctx_ws, ref, rtol=1e-12, atol=0.0)

    out = torch.full((3,), -1.0, dtype=torch.float64, device=dev)
    free0 = None
    for call in range(2):      # the shared accumulators must be cleared by every call
        rc = _call(lib, prec, obs.nrow, obs.nchan, 3, band, wt, out.data_ptr(), dev)
        assert rc == 0, lib.pfb_last_error(None)
        got = out.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-12, atol=0.0), (got, ref)
        torch.cuda.synchronize(dev)
        free = torch.cuda.mem_get_info(dev)[0]
        if call == 0:
            free0 = free
        else:
            assert free == free0        # no device allocation by the second call
        assert torch.cuda.current_device() == 0

    # host destinations (pinned and pageable), no weights
    pinned = torch.full((3,), -1.0, dtype=torch.float64).pin_memory()
    rc = _call(lib, prec, obs.nrow, obs.nchan, 3, band, None, pinned.data_ptr(), dev)
    assert rc == 0, lib.pfb_last_error(None)
    assert np.allclose(pinned.numpy(), ref_unit, rtol=1e-12, atol=0.0)
    pageable = np.full(3, -1.0)
    rc = _call(lib, prec, obs.nrow, obs.nchan, 3, band, wt, pageable.ctypes.data, dev)
    assert rc == 0, lib.pfb_last_error(None)
    assert np.allclose(pageable, ref, rtol=1e-12, atol=0.0)

    # errors: too many bands, a band id outside [0, nband), weights in host memory
    rc = _call(lib, prec, obs.nrow, obs.nchan, 33, band, wt, out.data_ptr(), dev)
    assert rc == -1 and b"maximum" in lib.pfb_last_error(None)
    bad = torch.tensor([0, 0, 1, 2, 3, 2], dtype=torch.int32, device=dev)
    rc = _call(lib, prec, obs.nrow, obs.nchan, 3, bad, wt, out.data_ptr(), dev)
    assert rc == -1 and b"outside" in lib.pfb_last_error(None)
    wt_host = torch.from_numpy(w)
    rc = _call(lib, prec, obs.nrow, obs.nchan, 3, band, wt_host, out.data_ptr(), dev)
    assert rc == -1 and b"device" in lib.pfb_last_error(None)
    # and the next valid call is correct again
    rc = _call(lib, prec, obs.nrow, obs.nchan, 3, band, wt, out.data_ptr(), dev)
    assert rc == 0 and np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0.0)


_FIRST_CALL = r"""
import ctypes, sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2101_08072_gb300 import _lib
lib = _lib.load()
dev = torch.device("cuda", 0)
band = torch.tensor([0, 1, 1, 0], dtype=torch.int32, device=dev)
w = torch.arange(1, 13, dtype=torch.float32, device=dev).reshape(3, 4)
out = np.zeros(2)
for _ in range(2):
    rc = lib.pfb_wsum_static(0, 0, 3, 4, 2, ctypes.c_void_p(band.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                             ctypes.c_void_p(out.ctypes.data),
                             ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    assert rc == 0, lib.pfb_last_error(None)
    # band 0: channels 0 and 3, band 1: channels 1 and 2 of rows (1..4), (5..8), (9..12)
    assert out.tolist() == [1 + 4 + 5 + 8 + 9 + 12, 2 + 3 + 6 + 7 + 10 + 11], out
print("ok")
"""


def test_wsum_static_first_call_in_fresh_process():
    """The first library call of a process is pfb_wsum_static (its one-time lookup of the
    accumulators' device address, before any other entry point has touched the device)."""
    _lib()
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
