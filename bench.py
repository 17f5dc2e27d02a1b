#!/usr/bin/env python
"""Throughput of the exact Hessian-vector product R^dagger Sigma^-1 R x on the
MeerKAT-like wide-field continuum workload (64 antennas / 2016 baselines x 450
integrations = 907,200 rows, 256 channels over 0.856-1.712 GHz in 4 imaging
bands, 4096^2 pixels of 1.5 arcsec, FP32 data with FP64 coordinates/phases,
epsilon = 3e-5), in million visibilities per second.

One step = one pfb_hessian call (R, weights, R^dagger over all 4 bands).
Inputs are synthetic and seeded, resident in HBM before the timed region; every
step touches tens of GB of w-plane stacks, far more than the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) each rank runs an independent replica of the workload
(the path shards only with an image all-reduce, which this program does not use);
value is the sum over ranks, timed as the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mvis/s for R^dagger Sigma^-1 R x (FP32, eps<=3e-5 vs FP64)"
UNIT = "Mvis/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--eps", type=float, default=3e-5)
    ap.add_argument("--ntime", type=int, default=450, help="integrations (907,200 rows at 450)")
    ap.add_argument("--npix", type=int, default=4096)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--serve", action="store_true",
                    help="serving workload instead: Poisson stream of mixed-size pfb-clean requests")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-max-pix", type=int, default=4096)
    ap.add_argument("--serve-max-rows", type=int, default=1_000_000)
    ap.add_argument("--serve-fp64-max-rows", type=int, default=200_000,
                    help="row cap of the FP64 requests (eps 1e-9, 1331 taps per visibility in FP64: "
                         "a 1e6-row FP64 request alone takes minutes)")
    ap.add_argument("--clean", action="store_true",
                    help="full pfb-clean workload instead: PSF, dirty image and --clean-outer steps (pfb_clean)")
    ap.add_argument("--clean-npix", type=int, default=8192)
    ap.add_argument("--clean-rows", type=int, default=2_200_000)
    ap.add_argument("--clean-chan", type=int, default=64)
    ap.add_argument("--clean-outer", type=int, default=20)
    ap.add_argument("--clean-pd", type=int, default=10, help="primal-dual iterations per step")
    ap.add_argument("--clean-cg", type=int, default=10, help="CG iterations per step")
    ap.add_argument("--clean-gamma", type=float, default=0.5,
                    help="step size; at the 8192^2 field gamma = 1 diverges slowly: the PSF-based preconditioner "
                         "underestimates the wide-field Hessian in some directions by more than 2x")
    ap.add_argument("--clean-sigma", type=float, default=1e-3)
    ap.add_argument("--clean-lambda", type=float, default=1e-4)
    ap.add_argument("--clean-basis", type=int, default=0b1111111, help="basis mask (bit 0 Dirac, 1..6 db1..db6)")
    ap.add_argument("--clean-safe-gamma", action="store_true",
                    help="cap gamma at 1.9 / lambda_max(U^-1 H), estimated by power iteration (PFB_STEP_SAFE_GAMMA)")
    ap.add_argument("--clean-tol", type=float, default=0.0,
                    help="stop at this relative update (0: run --clean-outer steps)")
    ap.add_argument("--facets", type=int, default=0,
                    help="faceted Hessian instead: the image split into F x F facets (R = sum of the facets' R)")
    ap.add_argument("--facets-wide", action="store_true",
                    help="with --facets: the full pfb-clean field (8192^2, 64 channels, --clean-rows rows)")
    ap.add_argument("--no-fp64", action="store_true",
                    help="skip the FP64 path (eps 1e-9) on the same workload (run by default, after the rest)")
    ap.add_argument("--no-rows", action="store_true", help="skip the per-entry-point timings")
    return ap.parse_args()


def workload(args):
    from paper_2101_08072_gb300 import synth
    obs = synth.meerkat_like_observation(ntime=args.ntime, nx=args.npix, ny=args.npix)
    rng = np.random.default_rng(2)
    bf = synth.band_centre_freqs(obs.freq, obs.band_of_chan, obs.nband)
    x = synth.point_source_image(rng, obs.nband, obs.nx, obs.ny, 1000, flux="pareto", fmin=1e-3, fmax=1.0,
                                 spectral=True, band_freqs=bf)
    return obs, x


def config(args, obs):
    return {"workload": f"MeerKAT-like wide-field Hessian: {obs.nrow} rows x {obs.nchan} channels, "
                        f"{obs.nband} bands, {obs.nx}x{obs.ny} image at 1.5 arcsec, eps {args.eps:g}",
            "rows": obs.nrow, "channels": obs.nchan, "bands": obs.nband, "image": [obs.nx, obs.ny],
            "visibilities": obs.nvis, "epsilon": args.eps, "precision": args.prec,
            "l2": "inputs larger than L2 (w-plane stacks of several GB per band)",
            "sources": 1000}


# ------------------------------------------------------------------ clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ measured traffic
# sources that shape the gridding and degridding kernels and their item order (a profiled traffic
# figure is only valid for them)
TRAFFIC_SOURCES = ["common.cuh", "ctx.cuh", "plan.cu", "wstack.cu"]


def source_digest() -> str:
    """Digest of the sources of the profiled kernels."""
    import hashlib
    d = hashlib.sha256()
    src = os.path.join(ROOT, "paper_2101_08072_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        d.update(open(os.path.join(src, f), "rb").read())
    return d.hexdigest()[:16]


def profiled_traffic(group: str):
    """DRAM bytes (read + write) per launch of a kernel group, from profiles/traffic.json,
    or None when absent or taken on different sources."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    e = t.get(group)
    if not e or e.get("source_digest") != source_digest():
        return None
    return e.get("bytes_per_launch")


# ------------------------------------------------------------------ per-row timings
def time_rows(ctx, lib, g, obs, uvw, freq, band, x, wgt, stream, dev, reps=2):
    import torch
    from paper_2101_08072_gb300 import StepParams

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    nvis = obs.nvis
    vis = torch.empty((obs.nrow, obs.nchan), dtype=torch.complex64, device=dev)
    out = {}
    ms = timed(lambda: ctx.pfb_degrid(g, uvw, freq, band, x, out=vis))
    out["R (pfb_degrid)"] = {"ms": ms, "Mvis/s": nvis / ms / 1e3}
    img = torch.empty_like(x)
    ms = timed(lambda: ctx.pfb_grid(g, uvw, freq, band, vis, wgt, out=img))
    out["R^dagger Sigma^-1 (pfb_grid)"] = {"ms": ms, "Mvis/s": nvis / ms / 1e3}
    ms = timed(lambda: ctx.pfb_dirty(g, uvw, freq, band, vis, wgt, out=img))
    out["dirty (pfb_dirty)"] = {"ms": ms, "Mvis/s": nvis / ms / 1e3}
    psf = torch.empty((obs.nband, 2 * obs.nx, 2 * obs.ny), dtype=x.dtype, device=dev)
    ms = timed(lambda: ctx.pfb_psf(g, uvw, freq, band, wgt, out=psf))
    out["PSF (pfb_psf, 2x field)"] = {"ms": ms, "Mvis/s": nvis / ms / 1e3}
    ms = timed(lambda: ctx.pfb_psf_conv(g, psf, x, out=img))
    # algorithmic bytes: read x, write y, read the cached half spectrum of the 2x grid
    b = obs.nband * (obs.nx * obs.ny * 8 + (2 * obs.nx) * (obs.ny + 1) * 8)
    out["PSF convolution (pfb_psf_conv)"] = {"ms": ms, "GB/s": b / ms / 1e6}
    _, ws = ctx.pfb_dirty(g, uvw, freq, band, vis, wgt, out=img)
    prm = StepParams(gamma=1.0, sigma=1e-3, lam=1e-4, cg_iters=10, pd_iters=10, basis_mask=1)
    xs = torch.zeros_like(x)
    dual = torch.zeros((1,) + tuple(x.shape), dtype=x.dtype, device=dev)
    ms = timed(lambda: ctx.pfb_step(g, prm, uvw, freq, band, wgt, img, psf, ws, xs, dual, stats=False))
    out["pfb_step (1 Hessian, 10 CG, 10 primal-dual, Dirac)"] = {"ms": ms, "Mvis/s": nvis / ms / 1e3}
    prm7 = StepParams(gamma=1.0, sigma=1e-3, lam=1e-4, cg_iters=10, pd_iters=10, basis_mask=0b1111111, nlevel=3)
    dual7 = torch.zeros((7,) + tuple(x.shape), dtype=x.dtype, device=dev)
    ms = timed(lambda: ctx.pfb_step(g, prm7, uvw, freq, band, wgt, img, psf, ws, xs, dual7, stats=False))
    out["pfb_step (10 CG, 10 primal-dual, Dirac + db1..db6)"] = {"ms": ms}
    return out


# ------------------------------------------------------------------ multi-rank helpers
def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (the slowest rank times the job)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput in millions of units per second: every rank processes
    units_per_rank (independent replicas), timed by the slowest rank."""
    return world * units_per_rank / (ms_max * 1e-3) / 1e6


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(obs, x, wgt_rows, rows, pix):
    """Time the FP64 oracle on a bounded sample of the Hessian: R x on `rows`
    (all channels, all sources) and R^dagger of the weighted result at `pix`.
    Returns (Mvis/s extrapolated to a full-image Hessian, seconds, threads)."""
    import oracle
    sub_uvw = obs.uvw[rows]
    t0 = time.perf_counter()
    v = oracle.degrid(sub_uvw, obs.freq, obs.band_of_chan, x, obs.dl, obs.dm)
    t1 = time.perf_counter()
    img = oracle.grid(sub_uvw, obs.freq, obs.band_of_chan, v, wgt_rows, obs.nx, obs.ny, obs.dl, obs.dm,
                      obs.nband, pix=pix)
    t2 = time.perf_counter()
    nvis = len(rows) * obs.nchan
    npix_total = obs.nband * obs.nx * obs.ny
    # R^dagger at one pixel of band b reads only band b's channels: scale by pixels per band
    sec_per_vis = (t1 - t0) / nvis + (t2 - t1) / nvis * (npix_total / len(pix))
    return 1e-6 / sec_per_vis, t2 - t0, oracle.num_threads(), (v, img)


def cpu_baseline(obs, x, wgt_np_fn, n_rows=24576, n_pix=6144, seed=5, want_sample=False):
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(obs.nrow, n_rows, replace=False))
    pix = np.sort(rng.choice(obs.nband * obs.nx * obs.ny, n_pix, replace=False))
    wrows = wgt_np_fn(rows)
    value, secs, threads, (v, img) = oracle_sample(obs, x, wrows, rows, pix)
    info = {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"FP64 direct sum: R x on {n_rows} random rows x {obs.nchan} channels (1000 sources), "
                      f"R^dagger at {n_pix} random pixels; cost extrapolated linearly to the full "
                      f"{obs.nband}x{obs.nx}^2 Hessian ({secs:.1f} s of CPU work)"}
    if want_sample:
        return info, {"rows": rows, "pix": pix, "wgt": wrows, "vis": v, "img": img}
    return info


def accuracy(ctx, g, obs, uvw, freq, band, x, smp, dev, rdt):
    """Relative L2 error of the GPU operators against the FP64 oracle on its sample: R x at the
    sampled rows (all channels), taken from one pfb_degrid of the whole workload, and R^dagger
    Sigma^-1 of the oracle's visibilities of those rows (with their weights) at the sampled pixels,
    from pfb_grid on the same rows.  The error bound epsilon applies to each."""
    import torch
    cdt = torch.complex64 if rdt == torch.float32 else torch.complex128
    vis = ctx.pfb_degrid(g, uvw, freq, band, x)
    rows_t = torch.from_numpy(smp["rows"]).to(dev)
    v_gpu = vis.index_select(0, rows_t).cpu().numpy().astype(np.complex128)
    del vis
    v_or = smp["vis"]
    e_r = float(np.linalg.norm(v_gpu - v_or) / np.linalg.norm(v_or))
    sub_uvw = uvw.index_select(0, rows_t).contiguous()
    img = ctx.pfb_grid(g, sub_uvw, freq, band, torch.from_numpy(v_or).to(dev, cdt),
                       torch.from_numpy(smp["wgt"]).to(dev, rdt))
    got = img.reshape(-1).index_select(0, torch.from_numpy(smp["pix"]).to(dev)).cpu().numpy().astype(np.float64)
    ref = smp["img"]
    e_g = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return {"R": e_r, "R_dagger": e_g, "epsilon": g.epsilon,
            "sample": f"R x at {len(smp['rows'])} random rows x {obs.nchan} channels; R^dagger Sigma^-1 of the "
                      f"oracle's visibilities of those rows at {len(smp['pix'])} random pixels"}


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    obs, x = workload(args)
    wrng = np.random.default_rng(9)

    def wgt(rows):
        return wrng.uniform(0.5, 1.5, (len(rows), obs.nchan))

    vals = []
    info = None
    for i in range(args.warmup + args.steps):
        info = cpu_baseline(obs, x, wgt, n_rows=2048, n_pix=1024, seed=100 + i)
        if i >= args.warmup:
            vals.append(info["value"])
    value = statistics.median(vals)
    ms = obs.nvis / (value * 1e6) * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)", "impl": "reference",
            "config": config(args, obs),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": info["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context, Geometry, _lib

    obs, x_np = workload(args)
    rdt = torch.float32 if args.prec == "f32" else torch.float64
    uvw = torch.from_numpy(obs.uvw).to(dev)
    freq = torch.from_numpy(obs.freq).to(dev)
    band = torch.from_numpy(obs.band_of_chan.astype(np.int32)).to(dev)
    x = torch.from_numpy(x_np).to(dev, rdt)
    gen = torch.Generator(device=dev)
    gen.manual_seed(9)
    wgt = torch.empty((obs.nrow, obs.nchan), dtype=rdt, device=dev).uniform_(0.5, 1.5, generator=gen)
    y = torch.empty_like(x)
    g = Geometry(nx=obs.nx, ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=args.eps)
    ctx = Context(local)
    lib = _lib.load()
    stream = torch.cuda.current_stream(dev)

    def step():
        ctx.pfb_hessian(g, uvw, freq, band, x, wgt, out=y)

    t_plan = time.perf_counter()
    step()
    torch.cuda.synchronize(dev)
    t_plan = time.perf_counter() - t_plan
    for _ in range(max(0, args.warmup - 1)):
        step()
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = Clocks(local)
    barrier()
    clocks.start()
    lib.pfb_timing(ctx.h, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # per-kernel totals recorded by the library on the same stream
    import ctypes
    names = ctypes.create_string_buffer(4096)
    lib.pfb_timing_names(ctx.h, names, 4096)
    kern = {}
    for nm in [n for n in names.value.decode().split(",") if n and n != "w_planes"]:   # w_planes: a count
        L, T, B = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        lib.pfb_timing_read(ctx.h, nm.encode(), ctypes.byref(L), ctypes.byref(T), ctypes.byref(B))
        kern[nm] = {"launches": L.value, "ms": T.value, "bytes": B.value}
    L, T, B = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    lib.pfb_timing_read(ctx.h, b"*", ctypes.byref(L), ctypes.byref(T), ctypes.byref(B))
    own_launches = L.value
    lib.pfb_timing(ctx.h, 0)

    ms = max_over_ranks(ms, world, dev)
    value = job_throughput(obs.nvis, world, ms)

    # ---- end to end through the public API with host buffers (pfb_hessian_host: the library copies the
    # inputs in and the result out every step, overlapped with the computation)
    e2e = None
    if not args.no_e2e:
        h_uvw = uvw.cpu().pin_memory()
        h_freq = freq.cpu().pin_memory()
        h_band = band.cpu().pin_memory()
        h_wgt = wgt.cpu().pin_memory()
        h_x = x.cpu().pin_memory()
        h_y = torch.empty(y.shape, dtype=rdt, pin_memory=True)
        bi = sum(t.numel() * t.element_size() for t in (h_uvw, h_freq, h_band, h_wgt, h_x))
        bo = h_y.numel() * h_y.element_size()
        barrier()
        ctx.pfb_hessian_host(g, h_uvw, h_freq, h_band, h_x, h_wgt, out=h_y)   # plan on the host arrays' copies
        torch.cuda.synchronize(dev)
        lib.pfb_timing(ctx.h, 1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps + 1)]
        ev[0].record(stream)
        for i in range(args.e2e_steps):
            ctx.pfb_hessian_host(g, h_uvw, h_freq, h_band, h_x, h_wgt, out=h_y)
            ev[i + 1].record(stream)
        barrier()
        ems = max_over_ranks(ev[0].elapsed_time(ev[-1]) / args.e2e_steps, world, dev)
        # per call and kernel groups of the host-buffer calls, for the log (stderr)
        per_call = [round(ev[i].elapsed_time(ev[i + 1]), 2) for i in range(args.e2e_steps)]
        e2e_k = {nm: round(v / args.e2e_steps, 3) for nm, v in kernel_totals(ctx).items()}
        lib.pfb_timing(ctx.h, 0)
        print(f"e2e: {ems:.2f} ms per call (calls: {per_call}); kernel groups (ms per call): {e2e_k}",
              file=sys.stderr)
        e2e = {"value": job_throughput(obs.nvis, world, ems), "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo}

    # ---- roofline of the dominant kernel group (traffic from the committed DRAM capture
    # of that kernel, when its source has not changed since)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    dom = max(kern.items(), key=lambda kv: kv[1]["ms"]) if kern else None
    roof = None
    if dom:
        nm, d = dom
        per_launch_ms = d["ms"] / max(d["launches"], 1)
        per_launch_bytes = d["bytes"] / max(d["launches"], 1)
        gbs = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9
        roof = {"kernel": nm, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "peak_source": peak_src, "traffic": profiled_traffic(nm),
                "share_of_step": d["ms"] / (ms * args.steps) if ms > 0 else None}
        if nm in ("grid_tiles", "degrid_tiles", "gather"):
            # The tile kernels are arithmetic scatters/gathers: W^2 W_w complex-by-real
            # multiply-adds per visibility (4 W^2 W_w flops), against the FP32 FMA peak of
            # the SMs (2 flops x 128 lanes x SMs x maximum SM clock).
            W = lib.pfb_kernel_support(args.eps, _lib.PFB_F32 if args.prec == "f32" else _lib.PFB_F64)
            flops = obs.nvis * 4.0 * W * W * W * args.steps / max(d["launches"], 1)
            props = torch.cuda.get_device_properties(dev)
            sm_mhz = peaks.get("sm_max_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
            peak_tf = 2.0 * 128 * props.multi_processor_count * sm_mhz * 1e6 / 1e12
            tf = flops / (per_launch_ms * 1e-3) / 1e12
            roof.update({"bound": "alu", "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s", "frac": tf / peak_tf,
                         "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x "
                                        f"{sm_mhz:.0f} MHz",
                         "algorithmic": f"4 W^2 W_w flop per visibility, W = W_w = {W}",
                         "hbm": {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                                 "peak_source": peak_src}})

    # ---- every entry point of the path on the same workload (one warm call, then timed calls)
    rows = None
    if not args.no_rows:
        rows = time_rows(ctx, lib, g, obs, uvw, freq, band, x, wgt, stream, dev)

    # ---- the oracle on the host cores (bounded sample), and the GPU operators' error on that sample
    cpu, acc = None, None
    if rank == 0 and world == 1:
        wnp = wgt.cpu().numpy().astype(np.float64)
        if args.no_cpu:
            _, smp = cpu_baseline(obs, x_np, lambda rows: wnp[rows], n_rows=1024, n_pix=256, want_sample=True)
        else:
            cpu, smp = cpu_baseline(obs, x_np, lambda rows: wnp[rows], want_sample=True)
        acc = accuracy(ctx, g, obs, uvw, freq, band, x, smp, dev, rdt)

    # ---- the FP64 path on the same workload (eps 1e-9), for the FP32-vs-FP64 comparison; last,
    # after the FP32 plans have given their memory back
    fp64 = None
    if not args.no_fp64 and args.prec == "f32":
        try:
            ctx.pfb_plan_reset()
            x64 = x.double()
            w64 = wgt.double()
            y64 = torch.empty_like(x64)
            g64 = Geometry(nx=obs.nx, ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=1e-9)
            t64 = time.perf_counter()
            ctx.pfb_hessian(g64, uvw, freq, band, x64, w64, out=y64)
            torch.cuda.synchronize(dev)
            t64 = time.perf_counter() - t64
            h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0.record(stream)
            ctx.pfb_hessian(g64, uvw, freq, band, x64, w64, out=y64)
            h1.record(stream)
            torch.cuda.synchronize(dev)
            ms64 = h0.elapsed_time(h1)
            # the FP32 Hessian against the FP64 one (same x and weights)
            ctx.pfb_plan_reset()
            ctx.pfb_hessian(g, uvw, freq, band, x, wgt, out=y)
            torch.cuda.synchronize(dev)
            d32 = float(torch.linalg.vector_norm(y.double() - y64) / torch.linalg.vector_norm(y64))
            fp64 = {"value": obs.nvis / (ms64 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms64, "epsilon": 1e-9,
                    "steps": 1, "first_call_s_with_plan": t64, "fp32_over_fp64": value / (obs.nvis / ms64 / 1e3),
                    "rel_l2_fp32_vs_fp64_hessian": d32}
            del x64, w64, y64
        except Exception as e:   # reported, not fatal: the FP32 line stands on its own
            fp64 = {"error": f"{type(e).__name__}: {str(e)[:300]}"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.prec, "data": "synthetic (seeded)",
                "config": config(args, obs), "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": own_launches, "clocks": clk, "fp64_path": fp64, "rows": rows,
                "rel_l2": acc,
                "kernels": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                                "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                            for k, v in sorted(kern.items(), key=lambda kv: -kv[1]["ms"])},
                "plan_s": t_plan}
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ serving workload
def serve_requests(n, seed=3, max_pix=4096, max_rows=1_000_000, fp64_max_rows=200_000):
    """n requests, each an independent pfb-clean solve: image 512^2..4096^2, rows 1e4..1e6,
    channels 8..128, bands 1..4 (log-uniform), half FP32 at eps 1e-5 and half FP64 at
    eps 1e-9, 10 steps each.  Visibilities are noise-like (the solver's cost does not
    depend on their values); geometry from the MeerKAT-like array."""
    from paper_2101_08072_gb300 import StepParams, synth
    from paper_2101_08072_gb300.serve import Request
    rng = np.random.default_rng(seed)
    base = synth.meerkat_like_observation(ntime=450)
    out = []
    for i in range(n):
        npix = int(2 ** round(np.log2(synth.log_uniform_int(rng, 512, max_pix + 1))))
        nrow = int(min(synth.log_uniform_int(rng, 1e4, max_rows), base.nrow))
        nchan = int(synth.log_uniform_int(rng, 8, 129))
        nband = int(min(nchan, synth.log_uniform_int(rng, 1, 5)))
        prec = "f32" if i % 2 == 0 else "f64"
        if prec == "f64":
            nrow = min(nrow, fp64_max_rows)
        rows = np.sort(rng.choice(base.nrow, nrow, replace=False))
        freq = np.linspace(0.856e9, 1.712e9, nchan)
        cell = 1.5 * 4096 / npix * synth.ARCSEC
        vis = (rng.normal(size=(nrow, nchan)) + 1j * rng.normal(size=(nrow, nchan))).astype(
            np.complex64 if prec == "f32" else np.complex128)
        wgt = rng.uniform(0.5, 1.5, (nrow, nchan)).astype(np.float32 if prec == "f32" else np.float64)
        out.append(Request(uvw=base.uvw[rows], freq=freq, band_of_chan=synth.contiguous_bands(nchan, nband),
                           vis=vis, wgt=wgt, nx=npix, ny=npix, dl=cell, dm=cell, nband=nband,
                           epsilon=1e-5 if prec == "f32" else 1e-9, precision=prec, n_iter=10,
                           params=StepParams(gamma=1.0, sigma=1e-3, lam=1e-4, cg_iters=20, pd_iters=20)))
    return out


def run_serve(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300.serve import Server
    reqs = serve_requests(args.serve_requests, max_pix=args.serve_max_pix, max_rows=args.serve_max_rows,
                          fp64_max_rows=args.serve_fp64_max_rows)
    # offered load: a Poisson stream at 0.8 of the sequential capacity.  The service time of a
    # request is modelled as (seconds per visibility-step of its precision) x visibilities x
    # (steps + 3, for the dirty image and the PSF); the per-precision rate comes from the first
    # FP32 and the first FP64 request, each run alone.
    srv = Server(0, max_active=1)
    per_vis_step = {}
    for prec in ("f32", "f64"):
        r = next(q for q in reqs if q.precision == prec)
        t0 = time.perf_counter()
        try:
            srv.submit(r).result()
        except Exception:
            pass
        per_vis_step[prec] = (time.perf_counter() - t0) / (r.nvis * (r.n_iter + 3))
    srv.close()
    predicted = [per_vis_step[q.precision] * q.nvis * (q.n_iter + 3) for q in reqs]
    rate = 0.8 / max(float(np.mean(predicted)), 1e-3)
    from paper_2101_08072_gb300 import synth
    arrivals = synth.poisson_arrivals(np.random.default_rng(4), len(reqs), rate)
    srv = Server(0, max_active=8)
    t0 = time.perf_counter()
    futs = []
    for r, ta in zip(reqs, arrivals):
        while time.perf_counter() - t0 < ta:
            time.sleep(0.001)
        futs.append(srv.submit(r))
    errors = 0
    messages = []
    for f in futs:
        try:
            f.result()
        except Exception as e:
            errors += 1
            if len(messages) < 4:
                messages.append(f"{type(e).__name__}: {str(e)[:200]}")
    srv.close()
    m = srv.metrics()
    line = {"metric": "serving latency (pfb-clean requests, 10 steps each)", "value": m["p50_s"], "unit": "s",
            "higher_is_better": False, "p50_s": m["p50_s"], "p99_s": m["p99_s"], "mvis_per_s": m["mvis_per_s"],
            "completed": m["completed"], "errors": errors, "error_messages": messages, "requests": len(reqs),
            "arrival_rate_per_s": rate, "predicted_sequential_s": float(np.sum(predicted)),
            "data": "synthetic (seeded)", "n_gpus": 1,
            "config": {"workload": f"Poisson stream of mixed-size requests: 512^2-{args.serve_max_pix}^2, "
                                   f"1e4-{args.serve_max_rows:.0e} rows (FP64 requests capped at "
                                   f"{args.serve_fp64_max_rows:.0e}), 8-128 channels, 1-4 bands, "
                                   "half FP32 eps 1e-5 / half FP64 eps 1e-9, 10 steps each"},
            "requests_detail": [{"pix": q.nx, "rows": int(q.uvw.shape[0]), "chan": int(q.freq.shape[0]),
                                 "bands": q.nband, "prec": q.precision,
                                 "latency_s": (q.t_done - q.t_submit) if q.t_done else None}
                                for q in reqs]}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ full pfb-clean workload
def clean_workload(args):
    """Full pfb-clean at scale: clean_npix^2 pixels of 1.5 arcsec, 4 bands, clean_chan channels over
    0.856-1.712 GHz, clean_rows rows (the MeerKAT-like array x enough 8 s integrations, truncated),
    5000 Pareto point sources (1 mJy - 1 Jy, index 1.5, spectral indices) plus 20 extended Gaussian
    sources with FWHM 5-60 pixels."""
    from paper_2101_08072_gb300 import synth
    nbl = 64 * 63 // 2
    ntime = -(-args.clean_rows // nbl)
    obs = synth.meerkat_like_observation(ntime=ntime, nchan=args.clean_chan, nx=args.clean_npix,
                                         ny=args.clean_npix)
    obs = synth.subset_rows(obs, np.arange(args.clean_rows))
    rng = np.random.default_rng(5)
    bf = synth.band_centre_freqs(obs.freq, obs.band_of_chan, obs.nband)
    x = synth.point_source_image(rng, obs.nband, obs.nx, obs.ny, 5000, flux="pareto", fmin=1e-3, fmax=1.0,
                                 spectral=True, band_freqs=bf)
    x += synth.gaussian_blob_image(rng, obs.nband, obs.nx, obs.ny, 20, fwhm_px=(5.0, 60.0))
    return obs, x


def run_clean(args):
    """One pfb_clean call (PSF on the 2x field, dirty image, clean_outer exact-gradient steps with the
    Dirac + db1..db6 dictionary) on data V = R x_true + noise of per-component std 1/sqrt(W).
    Reports the wall time, the count of full R^dagger Sigma^-1 R applications and the per-kernel
    split from the library's CUDA-event timing."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context, Geometry, StepParams
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    obs, x_np = clean_workload(args)
    rdt, cdt = (torch.float32, torch.complex64) if args.prec == "f32" else (torch.float64, torch.complex128)
    eps = args.eps if args.prec == "f32" else 1e-9
    uvw = torch.from_numpy(obs.uvw).to(dev)
    freq = torch.from_numpy(obs.freq).to(dev)
    band = torch.from_numpy(obs.band_of_chan.astype(np.int32)).to(dev)
    xt = torch.from_numpy(x_np).to(dev, rdt)
    del x_np
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    wgt = torch.empty((obs.nrow, obs.nchan), dtype=rdt, device=dev).uniform_(0.5, 1.5, generator=gen)
    g = Geometry(nx=obs.nx, ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=eps)
    ctx = Context(0)
    vis = ctx.pfb_degrid(g, uvw, freq, band, xt)
    sd = torch.rsqrt(wgt)
    vis += torch.complex(torch.randn(vis.shape, dtype=rdt, device=dev, generator=gen) * sd,
                         torch.randn(vis.shape, dtype=rdt, device=dev, generator=gen) * sd).to(cdt)
    del sd
    ctx.pfb_plan_reset()
    prm = StepParams(gamma=args.clean_gamma, sigma=args.clean_sigma, lam=args.clean_lambda, cg_iters=args.clean_cg,
                     pd_iters=args.clean_pd, nlevel=3, basis_mask=args.clean_basis,
                     safe_gamma=args.clean_safe_gamma)
    torch.cuda.synchronize(dev)
    ctx.lib.pfb_timing(ctx.h, 1)
    t0 = time.perf_counter()
    r = ctx.pfb_clean(g, prm, uvw, freq, band, vis, wgt, max_outer=args.clean_outer, tol=args.clean_tol)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    kern = kernel_totals(ctx)
    ctx.lib.pfb_timing(ctx.h, 0)
    x = r["x"]
    model_err = float(torch.linalg.vector_norm(x - xt) / torch.linalg.vector_norm(xt))
    hist = r["history"]
    lmax, gamma_used = ctx.pfb_last_step_bound() if args.clean_safe_gamma else (None, args.clean_gamma)
    to_1pct = next((i + 1 for i, h in enumerate(hist) if h[1] <= 1e-2), None)
    line = {"metric": "full pfb-clean solve wall time", "value": wall, "unit": "s", "higher_is_better": False,
            "n_outer": r["n_outer"], "n_hessian": r["n_hessian"],
            "mvis_per_s_hessian_equivalent": r["n_hessian"] * obs.nvis / wall / 1e6,
            "objective_first_last": [float(hist[0, 0]), float(hist[-1, 0])] if len(hist) else None,
            "rel_update_last": float(hist[-1, 1]) if len(hist) else None,
            "steps_to_rel_update_1e-2": to_1pct, "gamma_used": gamma_used, "lambda_max_UinvH": lmax,
            "history": [[float(v) for v in h] for h in hist],
            "rel_error_vs_true_sky": model_err,
            "kernels_ms": {k: round(v, 2) for k, v in sorted(kern.items(), key=lambda kv: -kv[1])[:16]},
            "dtype": args.prec, "data": "synthetic (seeded)", "n_gpus": 1,
            "config": {"workload": f"full pfb-clean: {obs.nx}^2 image at 1.5 arcsec (PSF {2 * obs.nx}^2), "
                                   f"{obs.nband} bands, {obs.nchan} channels over 0.856-1.712 GHz, {obs.nrow} rows, "
                                   f"5000 point + 20 Gaussian sources, basis mask {args.clean_basis:#b}, "
                                   f"{args.clean_outer} outer steps ({args.clean_cg} CG, {args.clean_pd} "
                                   f"primal-dual iterations each), gamma {args.clean_gamma:g}, "
                                   f"sigma {args.clean_sigma:g}, lambda {args.clean_lambda:g}",
                       "visibilities": obs.nvis, "epsilon": eps, "precision": args.prec}}
    ctx.close()
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ faceted Hessian
def run_facets(args):
    """The Hessian of the MeerKAT-like workload with the image split into F x F facets, each
    an image of its own centred at (l0, m0): V = sum_f R_f x_f (the first facet writes the
    visibilities, the others accumulate into them), then R_f^dagger (W V) per facet.  It is
    timed against the whole-image Hessian on the same data and compared with it."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_08072_gb300 import Context, Geometry, _lib
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    obs, x_np = clean_workload(args) if args.facets_wide else workload(args)
    F = args.facets
    fx, fy = obs.nx // F, obs.ny // F
    uvw = torch.from_numpy(obs.uvw).to(dev)
    freq = torch.from_numpy(obs.freq).to(dev)
    band = torch.from_numpy(obs.band_of_chan.astype(np.int32)).to(dev)
    x = torch.from_numpy(x_np).to(dev, torch.float32)
    gen = torch.Generator(device=dev)
    gen.manual_seed(9)
    wgt = torch.empty((obs.nrow, obs.nchan), dtype=torch.float32, device=dev).uniform_(0.5, 1.5, generator=gen)
    ctx = Context(0)
    stream = torch.cuda.current_stream(dev)
    g_full = Geometry(nx=obs.nx, ny=obs.ny, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=args.eps)
    facets = []
    for i0 in range(0, obs.nx, fx):
        for j0 in range(0, obs.ny, fy):
            l0 = (i0 + fx // 2 - obs.nx // 2) * obs.dl
            m0 = (j0 + fy // 2 - obs.ny // 2) * obs.dm
            gf = Geometry(nx=fx, ny=fy, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=args.eps, l0=l0, m0=m0)
            ga = Geometry(nx=fx, ny=fy, dl=obs.dl, dm=obs.dm, nband=obs.nband, epsilon=args.eps, l0=l0, m0=m0,
                          flags=_lib.PFB_ACCUMULATE)
            facets.append((i0, j0, gf, ga, x[:, i0:i0 + fx, j0:j0 + fy].contiguous(),
                           torch.empty((obs.nband, fx, fy), dtype=torch.float32, device=dev)))
    vis = torch.empty((obs.nrow, obs.nchan), dtype=torch.complex64, device=dev)
    y_full = torch.empty_like(x)

    def faceted():
        for k, (i0, j0, gf, ga, xf, yf) in enumerate(facets):
            ctx.pfb_degrid(ga if k else gf, uvw, freq, band, xf, out=vis)
        for i0, j0, gf, ga, xf, yf in facets:
            ctx.pfb_grid(gf, uvw, freq, band, vis, wgt, out=yf)

    def full():
        ctx.pfb_hessian(g_full, uvw, freq, band, x, wgt, out=y_full)

    def timed(fn, n):
        fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    ms_full = timed(full, args.steps)
    ms_fac = timed(faceted, args.steps)
    # planes per facet and for the whole image, from the plane bytes the library records per forward plane
    # block (pruned transforms: "w_planes", one plane sweep; full-plane transforms: "fft_fwd", two sweeps)
    def planes(fn, nx, ny):
        ctx.lib.pfb_timing(ctx.h, 1)
        fn()
        import ctypes
        n, ms, by = ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_double(0)
        ctx.lib.pfb_timing_read(ctx.h, b"w_planes", ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by))
        sweeps = 1.0
        if by.value == 0:
            ctx.lib.pfb_timing_read(ctx.h, b"fft_fwd", ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by))
            sweeps = 2.0
        ctx.lib.pfb_timing(ctx.h, 0)
        return by.value / (sweeps * (2 * nx) * (2 * ny) * 8)
    pl_full = planes(lambda: ctx.pfb_degrid(g_full, uvw, freq, band, x, out=vis), obs.nx, obs.ny)
    pl_fac = [planes(lambda f=f: ctx.pfb_degrid(f[2], uvw, freq, band, f[4], out=vis), fx, fy) for f in facets]
    faceted()
    full()
    torch.cuda.synchronize(dev)
    y_fac = torch.empty_like(x)
    for i0, j0, gf, ga, xf, yf in facets:
        y_fac[:, i0:i0 + fx, j0:j0 + fy] = yf
    diff = float(torch.linalg.vector_norm(y_fac - y_full) / torch.linalg.vector_norm(y_full))
    line = {"metric": "faceted Hessian R^dagger Sigma^-1 R x", "value": obs.nvis / (ms_fac * 1e-3) / 1e6,
            "unit": "Mvis/s", "ms_per_step": ms_fac, "whole_image_ms_per_step": ms_full,
            "whole_image_mvis_per_s": obs.nvis / (ms_full * 1e-3) / 1e6,
            "w_planes_whole_image": pl_full, "w_planes_per_facet": pl_fac,
            "rel_l2_vs_whole_image": diff, "facets": F * F, "dtype": "f32", "data": "synthetic (seeded)",
            "n_gpus": 1, "steps": args.steps,
            "config": {"workload": f"{'full pfb-clean field' if args.facets_wide else 'MeerKAT-like'} Hessian "
                                   f"({obs.nrow} rows x {obs.nchan} channels), {obs.nx}^2 image as {F}x{F} facets "
                                   f"of {fx}x{fy}",
                       "visibilities": obs.nvis, "epsilon": args.eps}}
    ctx.close()
    print(json.dumps(line))
    return 0


def kernel_totals(ctx):
    """ms per kernel group recorded by the library's timing since it was enabled."""
    import ctypes
    buf = ctypes.create_string_buffer(1 << 14)
    ctx.lib.pfb_timing_names(ctx.h, buf, len(buf))
    out = {}
    for name in (nm for nm in buf.value.decode().split(",") if nm and nm != "w_planes"):
        n, ms = ctypes.c_int64(0), ctypes.c_double(0)
        ctx.lib.pfb_timing_read(ctx.h, name.encode(), ctypes.byref(n), ctypes.byref(ms), None)
        out[name] = ms.value
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    if args.clean:
        return run_clean(args)
    if args.facets:
        return run_facets(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
