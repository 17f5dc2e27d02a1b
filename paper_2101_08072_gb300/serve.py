"""Continuous-batching server for independent pfb-clean solves.

Each request is one imaging problem (its own geometry, rows, channels, bands and
precision) solved by `n_iter` preconditioned forward-backward steps (Eqs. 6-7):
dirty image and PSF once, then pfb_step repeatedly, with all state resident in
HBM between steps.  The scheduler thread

  * admits queued requests, in arrival order, whenever their HBM reservation fits
    the memory left by the active ones (a request larger than the whole budget is
    rejected);
  * sets an admitted request up (uploads, PSF, plan, dirty image) on a worker
    thread, so the scheduler keeps issuing the running requests' steps meanwhile;
    the library allocates and frees stream-ordered, so neither the set-up nor a
    completion stalls the other requests' work on the device;
  * keeps every admitted request on its own CUDA stream and libpfb context, and
    issues one step at a time per request, so the steps of different requests run
    concurrently on the device; a request admitted while others are mid-solve
    joins the rotation once its set-up is done (continuous batching, not a FIFO of
    whole solves);
  * completes a request when its last step's event has fired, returns its image,
    dual and per-step statistics through a Future, and records its latency
    (submit -> result).

Results do not depend on the mix: a request's kernels run on its own stream in
the same order as when it runs alone, so its outputs agree with a solo run up to
floating-point reassociation inside the reductions (within the library's
tolerances).

The scheduling logic (`Scheduler`) is separate from the executor so that
admission and ordering are testable without a GPU.
"""
from __future__ import annotations

import dataclasses
import math
import queue
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
from typing import Any, Callable

import numpy as np


@dataclasses.dataclass
class Request:
    """One pfb-clean solve.  Arrays are host numpy arrays (copied to the device at admission)."""
    uvw: np.ndarray            # [nrow, 3] float64
    freq: np.ndarray           # [nchan] float64
    band_of_chan: np.ndarray   # [nchan] int32
    vis: np.ndarray            # [nrow, nchan] complex
    wgt: np.ndarray            # [nrow, nchan] real
    nx: int
    ny: int
    dl: float
    dm: float
    nband: int
    epsilon: float = 1e-5
    precision: str = "f32"     # "f32" or "f64"
    n_iter: int = 10
    params: Any = None         # StepParams
    tag: Any = None
    # filled by the server
    id: int = -1
    t_submit: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0

    @property
    def nvis(self) -> int:
        return int(self.uvw.shape[0] * self.freq.shape[0])


def footprint_bytes(r: Request) -> int:
    """HBM reserved for a request: its data, images, the plan's item lists, item
    records and pixel tables, and w-plane stacks for the operator and the PSF grid (the
    library processes plane blocks within whatever budget it is given, so the
    stacks are sized for a handful of planes, not the whole stack)."""
    rs = 4 if r.precision == "f32" else 8
    cs = 2 * rs
    nvis = r.nvis
    data = nvis * (cs + rs) + r.uvw.nbytes + nvis * 4 * 2 + nvis * cs     # vis, wgt, uvw, items, Hessian scratch
    img = r.nband * r.nx * r.ny
    images = img * rs * 10 + 4 * img * rs * 2 + 4 * img * cs                # x, dual, dirty, CG vectors, PSF, spectra
    tables = img * 16 + 4 * img * 16 + 2 * (1 << 25) * 12                  # pixel tables, bucket offsets
    if r.precision == "f32":
        tables += int(1.4 * nvis) * 24                                    # per-item geometry records
    grid = 4 * r.nx * r.ny * cs                                             # one oversampled plane
    planes = 12 * grid + 4 * 12 * grid                                      # operator and PSF plane blocks + FFT work
    return int(1.15 * (data + images + tables + planes)) + (64 << 20)


class Scheduler:
    """Admission by HBM footprint, FIFO order, bounded number of active requests."""

    def __init__(self, budget_bytes: int, max_active: int = 8):
        self.budget = budget_bytes
        self.max_active = max_active
        self.pending: list[Request] = []
        self.active: dict[int, int] = {}     # id -> reserved bytes

    @property
    def used(self) -> int:
        return sum(self.active.values())

    def add(self, r: Request):
        self.pending.append(r)

    def admissible(self) -> list[Request]:
        """Requests to admit now, in arrival order; stops at the first that does not fit
        (no overtaking, so a large request cannot starve)."""
        out = []
        while self.pending and len(self.active) < self.max_active:
            r = self.pending[0]
            need = footprint_bytes(r)
            if self.used + need > self.budget:
                break
            self.pending.pop(0)
            self.active[r.id] = need
            out.append(r)
        return out

    def too_large(self) -> list[Request]:
        """Pending requests that can never fit the budget (rejected)."""
        bad = [r for r in self.pending if footprint_bytes(r) > self.budget]
        self.pending = [r for r in self.pending if footprint_bytes(r) <= self.budget]
        return bad

    def release(self, rid: int):
        self.active.pop(rid, None)


class _Slot:
    """Device state of one admitted request."""

    def __init__(self, req: Request, fut: Future, device: int, reserve: int):
        import torch

        from .ops import Context, Geometry, StepParams
        self.req, self.fut = req, fut
        self.dev = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(self.dev)
        self.ctx = Context(device, reserve)
        self.geom = Geometry(req.nx, req.ny, req.dl, req.dm, req.nband, req.epsilon)
        self.params = req.params or StepParams()
        self.step = 0
        self.stats: list[np.ndarray] = []
        self.event = None
        rdt = torch.float32 if req.precision == "f32" else torch.float64
        cdt = torch.complex64 if req.precision == "f32" else torch.complex128
        with torch.cuda.stream(self.stream):
            t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(self.dev, dt, non_blocking=False)
            self.uvw = t(req.uvw, torch.float64)
            self.freq = t(req.freq, torch.float64)
            self.band = t(req.band_of_chan.astype(np.int32), torch.int32)
            self.vis = t(req.vis, cdt)
            self.wgt = t(req.wgt, rdt)
            nb = bin(self.params.basis_mask).count("1")
            self.x = torch.zeros((req.nband, req.nx, req.ny), dtype=rdt, device=self.dev)
            self.dual = torch.zeros((nb, req.nband, req.nx, req.ny), dtype=rdt, device=self.dev)
            # PSF first (2x field), then its plan and plane block go before the image-sized
            # plan that the dirty image and the steps share is built
            self.psf, _ = self.ctx.pfb_psf(self.geom, self.uvw, self.freq, self.band, self.wgt)
            self.ctx.pfb_plan_reset()
            self.dirty, self.wsum = self.ctx.pfb_dirty(self.geom, self.uvw, self.freq, self.band, self.vis, self.wgt)

    def issue_step(self):
        import torch
        with torch.cuda.stream(self.stream):
            self.ctx.pfb_step(self.geom, self.params, self.uvw, self.freq, self.band, self.wgt, self.dirty,
                              self.psf, self.wsum, self.x, self.dual, stats=False)
            self.event = torch.cuda.Event()
            self.event.record(self.stream)
        self.step += 1

    def ready(self) -> bool:
        return self.event is None or self.event.query()

    def finish(self):
        import torch
        with torch.cuda.stream(self.stream):
            x = self.x.cpu().numpy()
            dual = self.dual.cpu().numpy()
        self.ctx.close()
        return {"x": x, "dual": dual, "wsum": self.wsum, "steps": self.step}


class Server:
    """Persistent request loop on one GPU (see module docstring)."""

    def __init__(self, device: int = 0, budget_bytes: int | None = None, max_active: int = 8,
                 slot_factory: Callable[..., Any] = _Slot):
        self.device = device
        if budget_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info(device)
            budget_bytes = int(0.8 * free)
        self.sched = Scheduler(budget_bytes, max_active)
        self.slot_factory = slot_factory
        self.inbox: queue.Queue = queue.Queue()
        self.futures: dict[int, Future] = {}
        self.latencies: list[float] = []
        self.vis_done = 0
        self._next_id = 0
        self._stop = threading.Event()
        self._t0 = None
        self._t_last = None
        self._setup_pool = ThreadPoolExecutor(max_workers=2, thread_name_prefix="pfb-admit")
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def submit(self, r: Request) -> Future:
        fut: Future = Future()
        r.id = self._next_id
        self._next_id += 1
        r.t_submit = time.perf_counter()
        self.futures[r.id] = fut
        self.inbox.put(r)
        return fut

    def close(self):
        self._stop.set()
        self.thread.join()
        self._setup_pool.shutdown(wait=True)

    def metrics(self) -> dict:
        lat = np.array(self.latencies)
        span = (self._t_last - self._t0) if self._t0 is not None and self._t_last is not None else float("nan")
        return {"completed": int(lat.size),
                "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "mvis_per_s": (self.vis_done / span / 1e6) if span and span > 0 else None}

    # ------------------------------------------------------------------ loop
    def _setup(self, r: Request, fut: Future, reserve: int):
        """Device set-up of an admitted request, on a worker thread."""
        if self.slot_factory is _Slot:
            import torch
            torch.cuda.set_device(self.device)
        return self.slot_factory(r, fut, self.device, reserve)

    def _loop(self):
        if self.slot_factory is _Slot:
            import torch
            torch.cuda.set_device(self.device)
        slots: dict[int, Any] = {}
        setting_up: dict[int, tuple] = {}   # id -> (set-up future, request future)
        while (not self._stop.is_set() or slots or setting_up or not self.inbox.empty()
               or self.sched.pending):
            while True:
                try:
                    r = self.inbox.get_nowait()
                except queue.Empty:
                    break
                self.sched.add(r)
            for r in self.sched.too_large():
                self.futures.pop(r.id).set_exception(
                    MemoryError(f"request {r.id} needs {footprint_bytes(r)} B, more than the server budget"))
            for r in self.sched.admissible():
                fut = self.futures.pop(r.id)
                r.t_admit = time.perf_counter()
                if self._t0 is None:
                    self._t0 = r.t_admit
                setting_up[r.id] = (self._setup_pool.submit(self._setup, r, fut, self.sched.active[r.id]), fut)
            for rid in list(setting_up):
                sf, fut = setting_up[rid]
                if not sf.done():
                    continue
                setting_up.pop(rid)
                try:
                    slots[rid] = sf.result()
                except Exception as e:   # failed set-up: report to the caller, free the reservation
                    self.sched.release(rid)
                    fut.set_exception(e)
            idle = True
            for rid in list(slots):
                s = slots[rid]
                if not s.ready():
                    continue
                idle = False
                try:
                    if s.step < s.req.n_iter:
                        s.issue_step()
                        continue
                    res = s.finish()
                except Exception as e:
                    slots.pop(rid)
                    self.sched.release(rid)
                    s.fut.set_exception(e)
                    continue
                slots.pop(rid)
                self.sched.release(rid)
                s.req.t_done = time.perf_counter()
                self._t_last = s.req.t_done
                self.latencies.append(s.req.t_done - s.req.t_submit)
                self.vis_done += s.req.nvis * s.req.n_iter
                s.fut.set_result(res)
            if idle:
                time.sleep(0.0005)
