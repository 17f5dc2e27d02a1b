"""The serving loop on the GPU: requests of different sizes and precisions run
concurrently (continuous batching) and each result equals the same request run
alone, within the library's tolerance."""
import numpy as np
import pytest

import oracle
from paper_2101_08072_gb300 import synth

pytestmark = pytest.mark.gpu


def _request(seed, nx, ny, nband, nchan, prec, n_iter=3):
    from paper_2101_08072_gb300 import StepParams
    from paper_2101_08072_gb300.serve import Request
    obs = synth.tiny_observation(seed=seed, nx=nx, ny=ny, nchan=nchan, nband=nband)
    rng = np.random.default_rng(seed)
    x = synth.point_source_image(rng, nband, nx, ny, 4)
    V = oracle.degrid(obs.uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    V = V + synth.complex_noise(rng, V.shape, 1e-4)
    w = rng.uniform(0.5, 1.5, V.shape)
    return Request(uvw=obs.uvw, freq=obs.freq, band_of_chan=obs.band_of_chan, vis=V, wgt=w, nx=nx, ny=ny,
                   dl=obs.dl, dm=obs.dm, nband=nband, epsilon=1e-5 if prec == "f32" else 1e-10,
                   precision=prec, n_iter=n_iter,
                   params=StepParams(gamma=1.0, sigma=1e-2, lam=1e-3, cg_iters=10, pd_iters=20))


def test_mix_equals_alone():
    import time

    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300.serve import Server
    specs = [(1, 64, 64, 1, 4, "f32"), (2, 96, 128, 2, 8, "f32"), (3, 64, 64, 1, 4, "f64"), (4, 128, 64, 1, 6, "f32")]
    alone = []
    for sp in specs:
        srv = Server(0, max_active=1)
        alone.append(srv.submit(_request(*sp)).result(timeout=300))
        srv.close()
    srv = Server(0, max_active=8)
    futs = [srv.submit(_request(*sp)) for sp in specs[:3]]
    time.sleep(0.05)
    futs.append(srv.submit(_request(*specs[3])))   # arrives while the others are running
    mixed = [f.result(timeout=300) for f in futs]
    srv.close()
    m = srv.metrics()
    assert m["completed"] == 4 and m["p50_s"] > 0 and m["p99_s"] >= m["p50_s"]
    for sp, a, b in zip(specs, alone, mixed):
        tol = 1e-5 if sp[-1] == "f32" else 1e-11
        assert a["steps"] == b["steps"] == 3
        assert np.linalg.norm(a["x"] - b["x"]) <= tol * max(np.linalg.norm(a["x"]), 1e-30), sp
