"""Host-side logic of the serving loop (no GPU): admission by HBM footprint in
arrival order, continuous admission while others run, rejection of requests
larger than the budget, and failures reported through the Future without
stopping the other requests (failures are made on the host)."""
import time

import numpy as np
import pytest

from paper_2101_08072_gb300.serve import Request, Scheduler, Server, footprint_bytes


def _req(n=64, nrow=100, nchan=4, nband=1, n_iter=3, tag=None):
    z = np.zeros
    return Request(uvw=z((nrow, 3)), freq=np.ones(nchan), band_of_chan=z(nchan, np.int32),
                   vis=z((nrow, nchan), np.complex64), wgt=z((nrow, nchan), np.float32),
                   nx=n, ny=n, dl=1e-5, dm=1e-5, nband=nband, n_iter=n_iter, tag=tag)


def test_footprint_grows_with_size():
    a, b = footprint_bytes(_req(64)), footprint_bytes(_req(512))
    assert b > a > 0
    c = footprint_bytes(_req(64, nrow=100000))
    assert c > a


def test_scheduler_admits_in_order_within_budget():
    small, big = _req(64), _req(1024)
    s = Scheduler(budget_bytes=footprint_bytes(small) * 2 + 10, max_active=8)
    for i, r in enumerate([small, big, _req(64)]):
        r.id = i
        s.add(r)
    got = s.admissible()
    assert [r.id for r in got] == [0]            # the big one blocks the queue (no overtaking)
    assert s.too_large() == [big] or footprint_bytes(big) <= s.budget
    s.release(0)


class FakeSlot:
    """Stand-in for the device state: each step takes a little host time."""
    def __init__(self, req, fut, device, reserve):
        if req.tag == "fail-setup":
            raise ValueError("bad request")
        self.req, self.fut, self.step = req, fut, 0
        self.t = time.perf_counter()

    def ready(self):
        return time.perf_counter() - self.t > 0.002

    def issue_step(self):
        if self.req.tag == "fail-step" and self.step == 1:
            raise RuntimeError("step failed")
        self.step += 1
        self.t = time.perf_counter()

    def finish(self):
        return {"steps": self.step, "tag": self.req.tag}


def test_server_continuous_batching_and_failures():
    budget = footprint_bytes(_req(64)) * 3
    srv = Server(budget_bytes=budget, max_active=4, slot_factory=FakeSlot)
    futs = [srv.submit(_req(64, n_iter=5, tag=i)) for i in range(3)]
    time.sleep(0.01)
    late = srv.submit(_req(64, n_iter=2, tag="late"))           # arrives while others run
    bad = srv.submit(_req(64, tag="fail-setup"))
    bad2 = srv.submit(_req(64, n_iter=3, tag="fail-step"))
    huge = srv.submit(_req(8192))                                 # can never fit
    res = [f.result(timeout=10) for f in futs]
    assert [r["steps"] for r in res] == [5, 5, 5]
    assert late.result(timeout=10)["tag"] == "late"
    with pytest.raises(ValueError):
        bad.result(timeout=10)
    with pytest.raises(RuntimeError):
        bad2.result(timeout=10)
    with pytest.raises(MemoryError):
        huge.result(timeout=10)
    srv.close()
    m = srv.metrics()
    assert m["completed"] == 4 and m["p99_s"] >= m["p50_s"] > 0
