"""Benchmark of the particle -> IFU cube forward model on GB300.

One step = one full forward (spaxel keys, sort, SSP lookup + Doppler
resampling + per-spaxel deposit, combine of split spaxels, PSF + LSF) of the
large galaxy workload: 2e7 star particles (30% Hernquist bulge + exponential
disk), SSP grid 50 ages x 10 metallicities x 3721 wavelengths stored in BF16
(FP32 arithmetic), IFU of 300 x 300 spaxels of 0.1 kpc x 3721 bins of 1.25 A
from 4750 A, Gaussian PSF (FWHM 1.5 spaxels) and LSF (sigma 1.2 A) -- the
largest single-GPU configuration. Metric: particle-wavelength deposits per
second (in-field particles x wavelength bins / step time), with p50/p99 cube
latency. The mid-size galaxy (1e6 particles, FP32 templates), the
differentiable step, bin means and the serving stream are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank forward-models its own galaxy on its own GPU
(independent problems, no data-path collective: weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-wavelength deposits/s and p50/p99 cube latency at stated rel err"
UNIT = "deposits/s"
FLOPS_PER_DEPOSIT = 16  # 4 SSP corners x 2 wavelength neighbours, one FMA each
REL_ERR_BOUND = {"f32": 1e-5, "bf16": 2e-3}
CSRC = os.path.join(ROOT, "paper_2412_08265_gb300", "csrc")
# sources of the deposit kernel's code: a recorded DRAM traffic figure holds
# only for the kernel built from the same sources
DEPOSIT_SOURCES = ("deposit.cu", "tile.cuh", "common.cuh")


def deposit_sources_sha() -> str:
    h = hashlib.sha256()
    for name in DEPOSIT_SOURCES:
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes (read + write) of one deposit launch of `workload`, from the
    ncu summary profiles/k_deposit_<workload>.md (its lines
    `dram_bytes_per_launch: <bytes>` and `deposit_sources_sha256: <hash>`),
    or None if there is none or it was taken from other kernel sources."""
    path = os.path.join(ROOT, "profiles", f"k_deposit_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None, None
    vals = {}
    for line in text.splitlines():
        line = line.strip().strip("`")
        for key in ("dram_bytes_per_launch", "deposit_sources_sha256"):
            if line.startswith(key + ":"):
                vals[key] = line.split(":", 1)[1].strip()
    if vals.get("deposit_sources_sha256") != deposit_sources_sha() or "dram_bytes_per_launch" not in vals:
        return None, os.path.relpath(path, ROOT)
    return float(vals["dram_bytes_per_launch"]), os.path.relpath(path, ROOT)


def measured_fp32_peak():
    """FP32 FMA peak measured on this device now (FFMA and packed FFMA2 chain
    benchmarks in the library; the larger is the denominator)."""
    from paper_2412_08265_gb300 import capi
    runs = []
    for packed in (False, True):
        f, per_clk, mhz = capi.rubix_measure_fp32_peak(packed)
        runs.append({"kind": "FFMA2" if packed else "FFMA", "tflops": f / 1e12, "fma_per_clk_per_sm": per_clk,
                     "sm_mhz": mhz})
    best = max(runs, key=lambda r: r["tflops"])
    return best, runs


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def whole_job(units: float, seconds: float, device=None):
    """Whole-job aggregate over the ranks of the default process group: the
    units all ranks processed and the slowest rank's time (a single process
    returns its own). Returns (units / seconds, units, seconds)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units / seconds, units, seconds
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(t.item()), float(u.item()), float(t.item())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample(wl, target_s: float, seed: int = 123, cores: int | None = None):
    """Time the oracle's deposit over a seeded set of spaxel neighbourhoods sized
    for roughly target_s seconds; returns (deposits/s, cores, description,
    centres, cube0 for the sample, key)."""
    import oracle
    tel = wl.telescope
    p = wl.particles
    cores = cores or os.cpu_count() or 1
    xp, yp, v = oracle.orient(p)
    key = oracle.spaxel_keys(xp, yp, tel)
    n_s = tel.nx * tel.ny
    counts = np.bincount(key, minlength=n_s + 1)[:n_s]
    rng = np.random.default_rng(seed)
    order = rng.permutation(n_s)

    def mask_for(cs):
        m = np.zeros(n_s, np.uint8)
        for s in cs:
            y, x = divmod(int(s), tel.nx)
            for yy in range(max(0, y - 3), min(tel.ny, y + 4)):
                m[yy * tel.nx + max(0, x - 3): yy * tel.nx + min(tel.nx, x + 4)] = 1
        return m

    # calibrate on a small sample
    cal = order[:4]
    m = mask_for(cal)
    t0 = time.perf_counter()
    oracle.deposit(key, v, p, wl.ssp, tel, mask=m, n_threads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    rate = counts[m == 1].sum() * tel.n_lambda / dt
    budget = rate * target_s
    cs, tot = [], 0
    m = np.zeros(n_s, np.uint8)
    for s in order:
        cs.append(s)
        m = mask_for(cs) if len(cs) % 8 == 0 else m
        tot = counts[mask_for(cs) == 1].sum() * tel.n_lambda if len(cs) % 8 == 0 else tot
        if tot >= budget or len(cs) >= n_s:
            break
    m = mask_for(cs)
    dep = int(counts[m == 1].sum()) * tel.n_lambda
    t0 = time.perf_counter()
    cube0 = oracle.deposit(key, v, p, wl.ssp, tel, mask=m, n_threads=cores)
    dt = time.perf_counter() - t0
    desc = (f"FP64 oracle deposit over {int(m.sum())} of {n_s} spaxels (7x7 neighbourhoods of "
            f"{len(cs)} seeded centres), {int(counts[m == 1].sum())} particles x {tel.n_lambda} bins")
    return dep / dt, cores, desc, np.array(cs, dtype=np.int32), cube0, dep, dt


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    from paper_2412_08265_gb300 import synth
    wl = synth.large_galaxy() if args.workload == "large" else synth.mid_galaxy(n=args.particles)
    times, deps = [], []
    per_step = args.ref_step_seconds or max(3.0, 60.0 / max(args.steps + args.warmup, 1))
    for i in range(args.warmup + args.steps):
        rate, cores, desc, _, _, dep, dt = oracle_sample(wl, per_step, seed=1000 + i)
        if i >= args.warmup:
            times.append(dt)
            deps.append(dep)
    value = float(sum(deps) / sum(times))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "n_particles": wl.particles.n,
                       "spaxels": f"{wl.telescope.nx}x{wl.telescope.ny}", "n_lambda": wl.telescope.n_lambda,
                       "ssp": "50x10x3721, FP64 (the oracle's own precision)",
                       "sample": "bounded spaxel subset per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# serving: a Poisson request stream through the continuous-batching server,
# against the same server restricted to one galaxy per launch and one request
# on the GPU at a time (sequential one-galaxy-per-launch)
# ---------------------------------------------------------------------------
SERVE_SPAXEL_KPC = 0.2


def _drive(torch, srv, dev, reqs, ins, arrivals, max_outstanding=48):
    """Submit request i at arrivals[i] seconds (host clock), poll to completion.
    The client holds at most max_outstanding requests (and their output cubes)
    at a time; a later submit still counts its latency from its arrival time.
    Returns per-request latency (arrival -> completion, s) and the makespan."""
    from paper_2412_08265_gb300 import capi, synth
    n = len(reqs)
    lat = np.zeros(n)
    done_t = np.zeros(n)
    pend = {}
    t0 = time.perf_counter() + 0.02
    i = 0
    while i < n or pend:
        now = time.perf_counter()
        while i < n and now >= t0 + arrivals[i] and len(pend) < max_outstanding:
            tel = synth.serving_telescope(reqs[i]["side"])
            out = torch.empty((tel.ny, tel.nx, tel.n_lambda), dtype=torch.float32, device=dev)
            t_sub = time.perf_counter()
            pend[srv.submit(tel, ins[i], out)] = (i, out, t_sub)
            i += 1
            now = time.perf_counter()
        for tk in list(pend):
            st, l = srv.poll(tk)
            if st == capi.RUBIX_ERR_NOT_READY:
                continue
            if st != capi.RUBIX_OK:
                raise RuntimeError(f"request failed with status {st}: {capi.last_error_message()}")
            j, out, t_sub = pend.pop(tk)
            done_t[j] = t_sub + l
            lat[j] = done_t[j] - (t0 + arrivals[j])
        nxt = (t0 + arrivals[i] - time.perf_counter()) if i < n else 1e9
        time.sleep(max(0.0, min(nxt, 1e-4)))
    return lat, float(done_t.max() - (t0 + arrivals[0]))


def run_serving(args, dev, ssp):
    import torch
    from paper_2412_08265_gb300 import synth
    from paper_2412_08265_gb300.serve import Server
    n_req = args.serve_requests
    reqs = synth.serving_requests(n_req, seed=4, rate_hz=1.0)
    unit_arrivals = np.array([r["arrival_s"] for r in reqs])  # Poisson at 1 Hz; rescaled below
    n_max = max(r["n"] for r in reqs)
    mothers = [synth.disk_3d_device(n_max, 9000 + g, dev) for g in range(4)]
    ins, dep, vox = [], [], []
    for i, r in enumerate(reqs):
        m = mothers[i % len(mothers)]
        d = {k: v[: r["n"]] for k, v in m.items()}
        d["preprojected"] = False
        d["inclination"] = r["inclination"]
        ins.append(d)
        # in-field particles (host-side tally for the deposit count; not timed)
        half = 0.5 * r["side"] * SERVE_SPAXEL_KPC
        x = d["x"].double()
        yp = d["y"].double() * math.cos(r["inclination"]) - d["z"].double() * math.sin(r["inclination"])
        n_in = int(((x >= -half) & (x < half) & (yp >= -half) & (yp < half)).sum())
        dep.append(n_in * 3721)
        vox.append(r["side"] ** 2 * 3721)
    dep, vox = np.array(dep, dtype=np.float64), np.array(vox, dtype=np.float64)
    torch.cuda.synchronize()
    wl_grid = synth.serving_telescope(40)
    budget = int(args.serve_budget_gb * (1 << 30))

    def server(slots, batch):
        return Server(ssp, wl_grid, hbm_budget_bytes=budget, max_slots=slots, max_batch=batch, device=dev)

    # Each timed run gets a server whose memory pool is first grown to its
    # steady state (a long-running server's): 2 x slots requests of the
    # stream, all at once, before the clock starts (the first requests after
    # start-up pay the pool's growth, which a running server has behind it).
    def warm_server(slots, batch):
        srv = server(slots, batch)
        w = list(range(min(max(8, 2 * slots), n_req)))
        _drive(torch, srv, dev, [reqs[j] for j in w], [ins[j] for j in w], np.zeros(len(w)))
        return srv, srv.stats()

    def since(srv, st0):
        st = srv.stats()
        return {"deposit_launches": st["deposit_launches"] - st0["deposit_launches"],
                "max_batch": st["max_batch"], "peak_bytes": st["peak_bytes"]}

    # sequential capacity: every request queued at t = 0
    res = {}
    for name, cfg in (("sequential", (1, 1)), ("served", (args.serve_slots, args.serve_batch))):
        srv, st0 = warm_server(*cfg)
        _, mk = _drive(torch, srv, dev, reqs, ins, np.zeros(n_req))
        st = since(srv, st0)
        srv.close()
        res[name] = {"saturated": {"deposits_per_s": float(dep.sum() / mk), "requests_per_s": n_req / mk,
                                   "makespan_s": mk, "deposit_launches": st["deposit_launches"],
                                   "max_batch": st["max_batch"]}}
    # Poisson arrivals at fixed rates: each load x the sequential capacity
    loads = [float(x) for x in args.serve_loads.split(",") if x.strip()]
    cap = res["sequential"]["saturated"]["requests_per_s"]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for rho in loads:
        arrivals = unit_arrivals / (rho * cap)
        key = f"poisson_rho{rho:g}"
        for name, cfg in (("sequential", (1, 1)), ("served", (args.serve_slots, args.serve_batch))):
            srv, st0 = warm_server(*cfg)
            lat, mk = _drive(torch, srv, dev, reqs, ins, arrivals)
            st = since(srv, st0)
            srv.close()
            res[name][key] = {"load_vs_sequential_capacity": rho, "arrival_rate_hz": rho * cap,
                              "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                              "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                              "mean_ms": 1e3 * float(lat.mean()), "max_ms": 1e3 * float(lat.max()),
                              "deposits_per_s": float(dep.sum() / mk), "requests_per_s": n_req / mk,
                              "deposit_launches": st["deposit_launches"], "max_batch": st["max_batch"],
                              "peak_bytes": st["peak_bytes"]}
    clk = clocks.stop()
    del ins, mothers
    res["classes"] = _serve_classes(torch, server, dev, args)
    return {"requests": n_req, "sequential_capacity_requests_per_s": cap, "loads_vs_sequential_capacity": loads,
            "particles": "log-uniform [1e4, 2e7] (prefixes of 4 device-drawn 3-D disks)",
            "cube_side": "uniform [40, 300] spaxels of 0.2 kpc x 3721 bins",
            "inclination": "uniform [0, 90] deg", "deposits_total": float(dep.sum()),
            "voxels_total": float(vox.sum()), "max_slots": args.serve_slots, "max_batch": args.serve_batch,
            "hbm_budget_bytes": budget, "latency": "arrival to completion seen by the client",
            "clocks": clk, **res}


def _serve_classes(torch, server, dev, args):
    """The two ends of the request mix, each as a saturated stream through the
    served configuration: small galaxies in large cubes (HBM-bound: the
    deposit writes every voxel, the PSF/LSF reads and writes it again, 12 B per
    voxel) and large galaxies in small cubes (the deposit's FP32 work, 16 flop
    per deposit); each with its fraction of the matching peak."""
    from paper_2412_08265_gb300 import synth
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    props = torch.cuda.get_device_properties(dev)
    fp32 = props.multi_processor_count * 128 * 2 * float(peaks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    out = {}
    for name, n_p, side, count in (("small_galaxy_large_cube", 10_000, 300, 24),
                                   ("large_galaxy_small_cube", 20_000_000, 40, 8)):
        d = synth.disk_3d_device(n_p, 7100 + side, dev)
        d["preprojected"] = False
        d["inclination"] = 0.5
        half = 0.5 * side * SERVE_SPAXEL_KPC
        x = d["x"].double()
        yp = d["y"].double() * math.cos(0.5) - d["z"].double() * math.sin(0.5)
        n_in = int(((x >= -half) & (x < half) & (yp >= -half) & (yp < half)).sum())
        reqs = [{"side": side} for _ in range(count)]
        srv = server(args.serve_slots, args.serve_batch)
        # the pool grown to its steady state first, as in run_serving
        _drive(torch, srv, dev, reqs, [d] * count, np.zeros(count))
        _, mk = _drive(torch, srv, dev, reqs, [d] * count, np.zeros(count))
        srv.close()
        deposits = float(count) * n_in * 3721
        voxels = float(count) * side * side * 3721
        gbs = 12.0 * voxels / mk / 1e9
        tfl = 16.0 * deposits / mk / 1e12
        out[name] = {"requests": count, "particles": n_p, "cube_side": side, "makespan_s": mk,
                     "requests_per_s": count / mk, "deposits_per_s": deposits / mk,
                     "hbm_gbs": gbs, "hbm_frac_of_measured": gbs / hbm,
                     "fp32_tflops": tfl, "fp32_frac": tfl / fp32}
        del d
    return out


# ---------------------------------------------------------------------------
# the other single-GPU workloads: the differentiable step (1e6 particles, loss
# 1/2 |cube - target|^2 against a cube of perturbed ages, metallicities and
# velocities) and the large galaxy (2e7 particles, BF16 templates)
# ---------------------------------------------------------------------------
def _events_ms(torch, fn, stream, steps, flush):
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in ev])


def run_extra(args, dev, flush, peak_tflops):
    import torch
    from paper_2412_08265_gb300 import synth
    stream = torch.cuda.current_stream(dev)
    out = {}
    sel = set(args.extra.split(","))
    wl = synth.mid_galaxy(n=args.particles, seed=1)
    if "mid_f32" in sel:
        out["mid_f32"] = _extra_mid_f32(args, dev, flush, stream, peak_tflops)
    if "differentiable" in sel:
        out["differentiable"] = _extra_differentiable(args, dev, flush, wl, stream)
    if "bin_means" in sel:
        out["bin_means"] = _extra_bin_means(args, dev, flush, wl, stream)
    return out


def _extra_differentiable(args, dev, flush, wl, stream):
    import torch
    from paper_2412_08265_gb300 import synth
    from paper_2412_08265_gb300.model import CubeModel
    tgt_p = synth.perturbed_target(wl.particles)
    model = CubeModel(wl.ssp, wl.telescope, "f32", max_particles=wl.particles.n, device=dev)
    target = model.forward(tgt_p).clone()
    d = model.device_particles(wl.particles)
    cube = torch.empty(model.cube_shape, dtype=torch.float32, device=dev)
    res = {}

    def step():
        model.forward(d, out=cube)
        g = cube - target                      # dL/dcube of 1/2 |cube - target|^2
        res["grads"] = model.backward(g, want_global=True)

    for _ in range(3):
        step()
    n_dep = model.stats()["deposits"]
    t_step = _events_ms(torch, step, stream, max(3, min(args.steps, 10)), flush)
    t_fwd = _events_ms(torch, lambda: model.forward(d, out=cube), stream, max(3, min(args.steps, 10)), flush)
    grads = res["grads"]
    ok = all(bool(torch.isfinite(x).all()) for x in grads[:4]) and bool(torch.isfinite(grads[4]).all())
    res = {
        "workload": "mid-disk-1e6p-150x150x3721-f32, loss 1/2|cube - target|^2, target: ages/Z x (1 + N(0, 0.1)), v + 20 km/s",
        "step_ms": float(np.median(t_step)), "forward_ms": float(np.median(t_fwd)),
        "backward_ms": float(np.median(t_step) - np.median(t_fwd)),
        "deposits_per_s_forward_plus_backward": 2.0 * n_dep / (float(np.median(t_step)) / 1e3),
        "grads_finite": ok}
    model.close()
    return res


def _extra_bin_means(args, dev, flush, wl, stream):
    """Mid-size workload with flux-conserving bin means (resample = 1)."""
    import torch
    from paper_2412_08265_gb300 import synth
    from paper_2412_08265_gb300.model import CubeModel
    tel_m = synth.Telescope(**{**wl.telescope.__dict__, "resample": 1})
    model = CubeModel(wl.ssp, tel_m, "f32", max_particles=wl.particles.n, device=dev)
    d = model.device_particles(wl.particles)
    cube = torch.empty(model.cube_shape, dtype=torch.float32, device=dev)
    for _ in range(3):
        model.forward(d, out=cube)
    st = model.stats()
    model.set_profiling(True)
    t = _events_ms(torch, lambda: model.forward(d, out=cube), stream, max(3, min(args.steps, 10)), flush)
    dep = model.profile_history("deposit")
    model.set_profiling(False)
    # the backward of the same forward, for a fixed cotangent
    g = torch.randn(model.cube_shape, generator=torch.Generator(device=dev).manual_seed(5), device=dev)
    model.forward(d, out=cube)
    for _ in range(2):
        model.backward(g)
    tb = _events_ms(torch, lambda: model.backward(g), stream, max(3, min(args.steps, 10)), flush)
    res = {
        "workload": "mid-disk-1e6p-150x150x3721-f32, resample = 1 (mean over each output bin)",
        "ms_per_step": float(np.median(t)), "deposit_ms": float(np.median(dep)),
        "deposits_per_s": st["deposits"] / (float(np.median(t)) / 1e3),
        "backward_ms": float(np.median(tb)),
        "slow_particle_tiles": st["slow_particle_tiles"]}
    model.close()
    return res


def _extra_mid_f32(args, dev, flush, stream, peak_tflops):
    """Mid-size galaxy, FP32 templates (1e6 particles, 150 x 150 x 3721)."""
    import torch
    from paper_2412_08265_gb300 import synth
    from paper_2412_08265_gb300.model import CubeModel
    wl = synth.mid_galaxy(n=args.particles, seed=1)
    model = CubeModel(wl.ssp, wl.telescope, "f32", max_particles=wl.particles.n, device=dev)
    d = model.device_particles(wl.particles)
    cube = torch.empty(model.cube_shape, dtype=torch.float32, device=dev)
    for _ in range(3):
        model.forward(d, out=cube)
    st = model.stats()
    model.set_profiling(True)
    t = _events_ms(torch, lambda: model.forward(d, out=cube), stream, max(5, min(args.steps, 20)), flush)
    dep = model.profile_history("deposit")
    psf = model.profile_history("psf_lsf")
    model.set_profiling(False)
    dep_s = float(np.mean(dep)) / 1e3
    traffic, tsrc = recorded_traffic(wl.name)
    res = {
        "workload": wl.name, "n_in_fov": st["n_in_fov"], "ms_per_step": float(np.median(t)),
        "p50_ms": float(np.percentile(t, 50)), "p99_ms": float(np.percentile(t, 99)),
        "deposits_per_s": st["deposits"] / (float(np.median(t)) / 1e3),
        "deposit_ms": 1e3 * dep_s, "psf_lsf_ms": float(np.median(psf)),
        "deposit_fp32_tflops": st["deposits"] * FLOPS_PER_DEPOSIT / dep_s / 1e12,
        "deposit_frac_of_measured_fp32": st["deposits"] * FLOPS_PER_DEPOSIT / dep_s / 1e12 / peak_tflops,
        "deposit_dram_bytes": traffic, "traffic_source": tsrc,
        "tile_bins": st["tile_w"], "age_bands": st["n_bands"]}
    model.close()
    return res


def _e2e(args, dev, wl, dtype, model, stream, deposits):
    """End to end through the C ABI with host buffers: page-locked particle
    arrays in, page-locked host cube out, every copy inside the timing. The
    headline figure is the server (rubix_serve_submit) with a few requests in
    flight; the synchronous single-handle call is reported beside it."""
    import torch
    from paper_2412_08265_gb300 import capi
    from paper_2412_08265_gb300.serve import Server
    p = wl.particles
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k), dtype=np.float32)).pin_memory()
            for k in ("x", "y", "v_los", "mass", "age", "Z")}
    h2d = sum(v.numel() * 4 for v in host.values())
    cube_bytes = int(np.prod(model.cube_shape)) * 4
    depth = 3 if cube_bytes < (1 << 30) else 2
    outs = [torch.empty(model.cube_shape, dtype=torch.float32).pin_memory() for _ in range(depth)]
    cp = model.c_particles({**{k: v.numpy() for k, v in host.items()}, "preprojected": True,
                            "inclination": 0.0}, on_device=False)
    for _ in range(2):
        capi.rubix_cube_forward(model.handle, cp, 0, 0.0, outs[0].data_ptr(), 0, stream.cuda_stream)
    k_single = max(3, min(args.steps, 8))
    t0 = time.perf_counter()
    for _ in range(k_single):
        capi.rubix_cube_forward(model.handle, cp, 0, 0.0, outs[0].data_ptr(), 0, stream.cuda_stream)
    t_single = (time.perf_counter() - t0) / k_single
    single = {"value": deposits / t_single, "ms_per_step": 1e3 * t_single,
              "api": "rubix_cube_forward, host buffers, one call at a time (the call returns after the copy)"}
    budget = max(16 << 30, 3 * depth * model_bytes_estimate(model))
    srv = Server(wl.ssp, wl.telescope, template_dtype=dtype, hbm_budget_bytes=budget, max_slots=depth, max_batch=1,
                 device=dev)
    din = {**host, "preprojected": True, "inclination": 0.0}

    def burst(k):
        tks = []
        for i in range(k):
            if i >= depth and srv.wait(tks[i - depth], 120.0) != 0:
                raise RuntimeError("served request failed: " + capi.last_error_message())
            tks.append(srv.submit(wl.telescope, din, outs[i % depth]))
        for t in tks[max(0, k - depth):]:
            if srv.wait(t, 120.0) != 0:
                raise RuntimeError("served request failed: " + capi.last_error_message())

    burst(2 * depth)
    k_srv = max(3 * depth, min(args.steps, 10) * (2 if depth == 3 else 1))
    t_bursts = []
    for _ in range(3):  # three timed bursts; the median is reported
        t0 = time.perf_counter()
        burst(k_srv)
        t_bursts.append((time.perf_counter() - t0) / k_srv)
    t_srv = float(np.median(t_bursts))
    srv.close()
    return {"value": deposits / t_srv, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(cube_bytes), "ms_per_step": 1e3 * t_srv,
            "api": f"rubix_serve_submit, host buffers (page-locked), {depth} requests in flight, "
                   f"median of 3 bursts of {k_srv} requests",
            "burst_ms_per_step": [1e3 * t for t in t_bursts], "single_call": single}


def model_bytes_estimate(model) -> int:
    return int(np.prod(model.cube_shape)) * 4 * 4


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    from __graft_entry__ import build
    build()
    from paper_2412_08265_gb300 import synth
    from paper_2412_08265_gb300.model import CubeModel

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    wl = synth.large_galaxy(seed=2 + rank) if args.workload == "large" else synth.mid_galaxy(n=args.particles,
                                                                                              seed=1 + rank)
    dtype = wl.template_dtype
    model = CubeModel(wl.ssp, wl.telescope, dtype, max_particles=wl.particles.n, device=dev)
    d = model.device_particles(wl.particles)
    out = torch.empty(model.cube_shape, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        model.forward(d, out=out)
    torch.cuda.synchronize()
    st = model.stats()
    n_in, deposits, launches_per_step = st["n_in_fov"], st["deposits"], st["kernel_launches"]
    # the FP32 roof of the deposit, measured on this device just before the timed steps
    peak, peak_runs = measured_fp32_peak()

    model.set_profiling(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device() if ws == 1 else local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.fill_(float(i))           # evict L2 between timed steps (outside the events)
        ev[i][0].record(stream)
        model.forward(d, out=out)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    dep_ms = model.profile_history("deposit")
    stage_med = {k: float(np.median(model.profile_history(k)[-args.steps:]))
                 for k in ("assign_sort", "setup_items", "deposit", "combine", "psf_lsf", "forward")}
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    # every rank forward-models its own galaxy: deposits summed over ranks,
    # time of the slowest rank
    value, _, total_s = whole_job(deposits * args.steps, float(step_ms.sum()) / 1e3, device=dev)
    n_in_all = whole_job(n_in * args.steps, 1.0, device=dev)[1]
    model.set_profiling(False)

    e2e = _e2e(args, dev, wl, dtype, model, stream, deposits) if rank == 0 else None

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel (deposit) ----
    dep_avg_s = float(np.mean(dep_ms)) / 1e3
    achieved = deposits * FLOPS_PER_DEPOSIT / dep_avg_s / 1e12
    traffic, traffic_src = recorded_traffic(wl.name)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak["tflops"], "unit": "TFLOP/s",
            "frac": achieved / peak["tflops"], "traffic": traffic,
            "kernel": "k_deposit", "kernel_ms": 1e3 * dep_avg_s,
            "peak_basis": (f"measured on this GPU before the timed steps: {peak['kind']} dependent-chain benchmark "
                           f"(rubix_measure_fp32_peak), {peak['fma_per_clk_per_sm']:.1f} FMA/clk/SM at "
                           f"{peak['sm_mhz']:.0f} MHz"),
            "peak_runs": peak_runs, "traffic_source": traffic_src,
            "deposits_per_launch": deposits, "flops_per_deposit": FLOPS_PER_DEPOSIT}

    # ---- CPU baseline: the oracle on a bounded sample, and the sampled rel err ----
    cpu = None
    rel = None
    if not args.no_cpu_baseline:
        import oracle
        rate, cores, desc, centres, cube0, dep, dt = oracle_sample(wl, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
        # the same oracle on one core, over a smaller sample
        rate1, _, desc1, _, _, _, _ = oracle_sample(wl, max(2.0, args.cpu_seconds / 3), seed=321, cores=1)
        cpu["single_core"] = {"value": rate1, "sample": desc1}
        ref = oracle.psf_lsf_at(cube0, wl.telescope, centres[: min(len(centres), 24)])
        got = out.reshape(-1, wl.telescope.n_lambda)[torch.from_numpy(centres[: min(len(centres), 24)]).long().to(dev)]
        got = got.cpu().numpy().astype(np.float64)
        rel = float(np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300))

    tel = wl.telescope
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(step_ms.mean()), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "n_particles": wl.particles.n, "n_in_fov": n_in,
                       "spaxels": f"{tel.nx}x{tel.ny}", "spaxel_kpc": tel.spaxel_size, "n_lambda": tel.n_lambda,
                       "ssp": f"50x10x3721 stored {dtype}, FP32 arithmetic",
                       "psf_fwhm_spaxels": tel.psf_fwhm, "lsf_sigma_A": tel.lsf_sigma,
                       "l2": "flushed between timed steps", "parallelism": f"replicas x{ws}"},
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "rel_err_bound": REL_ERR_BOUND[dtype], "rel_err_sampled": rel,
            "particles_per_s": n_in_all / total_s,
            "clocks": clk, "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "stage_ms_median": stage_med,
            "deposit_geometry": {"tile_bins": st["tile_w"], "slab_nodes": st["slab_w"], "age_bands": st["n_bands"]}}
    model.close()
    del d, out
    torch.cuda.empty_cache()
    if not args.no_extra:
        line["workloads"] = run_extra(args, dev, flush, peak["tflops"])
    if args.serve_requests > 0:
        line["serving"] = run_serving(args, dev, synth.mid_galaxy(n=1000, seed=1).ssp)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=None,
                    help="oracle work per step of --impl reference (default: about a minute in all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--particles", type=int, default=1_000_000,
                    help="particles of the mid-size galaxy (smaller only for profiler captures)")
    ap.add_argument("--workload", default="large", choices=["large", "mid"],
                    help="workload of the timed steps (large: the largest single-GPU configuration)")
    ap.add_argument("--extra", default="mid_f32,differentiable,bin_means",
                    help="comma-separated extra workloads reported under 'workloads'")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the differentiable-step and large-galaxy measurements")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests in the serving stream (0 = no serving run)")
    ap.add_argument("--serve-loads", default="0.5,0.9",
                    help="Poisson arrival rates, as fractions of the sequential path's capacity")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-batch", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
