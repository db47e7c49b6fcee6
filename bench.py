"""Benchmark: hexagonal cell-updates per second of the explicit finite-volume step on the
large carved catchment (4096 x 4096 hexagons, edge 5 m, 16.7 M cells, land-cover classes,
2 h double-peak storm, outlet hydrograph every 10 s), on GB300.

One bench step = one time step of the whole hot path over the raster (edge fluxes, rain,
implicit friction, state update, CFL reduction, ledger and clock on the device).

Arms:
  default            the CUDA path through the C ABI (libasx.so)
  --impl reference   the FP64 CPU oracle on the host cores (a bounded crop per step)

Prints one JSON line.  Under torchrun (N > 1) each rank runs an independent replica of
the workload ("replicas only"); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hex cell-updates/s"
UNIT = "cell-updates/s"
BYTES_PER_CELL = 32            # read m, v1, v2, z, theta + write m, v1, v2 (float32)
T_WARM = 2700.0                # start of the timed window: between the storm peaks [s]
REF_CROP = 384                 # reference arm: crop side (cells) per oracle step


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def max_over_ranks(vals, device):
    """Each value's maximum over the ranks of the process group (the slowest replica sets
    the job's time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t]


def job_rate(ws, cells, steps, seconds):
    """Whole-job cell-updates per second: every replica updates `cells` cells `steps`
    times; the job takes the slowest replica's time."""
    return ws * cells * steps / seconds


def _workload_config(sc, k, t_warm=T_WARM):
    return {"workload": f"carved catchment {sc.rows}x{sc.cols} hex, edge {sc.l:g} m, "
                        f"3 land-cover classes, double-peak storm, window from t={t_warm:.0f} s",
            "cells": sc.n, "rows": sc.rows, "cols": sc.cols, "steps_timed": k,
            "l2": f"device state {sc.n * 37 / 1e9:.2f} GB (8 state planes, bed, classes) > 129 MB L2 "
                  "(no flush needed)", "parallelism": "replicas"}


def run_cuda(args):
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2406_14933_gb300 import build as pb
    pb.build()
    from paper_2406_14933_gb300 import asx as A
    from paper_2406_14933_gb300 import inputs
    from paper_2406_14933_gb300.raster import Raster

    sc = inputs.carved_catchment(rows=args.rows, cols=args.cols)
    stream = torch.cuda.current_stream()
    R = Raster(sc, device=local, stream=stream.cuda_stream)
    R.run_until(args.t_warm)
    R.step(args.warmup)
    warm_steps = R.clock()[2]
    n = sc.n

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    # device-timed regions of exactly K steps each, inputs resident in HBM, repeated until
    # at least args.min_timed_s has been timed (so that the clock sampler sees the load);
    # the value is the median region, the spread is reported beside it
    regions = []
    barrier()
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        while True:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            R.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            regions.append(e0.elapsed_time(e1))
            if sum(regions) >= 1e3 * args.min_timed_s or len(regions) >= args.max_regions:
                break
        torch.cuda.nvtx.range_pop()
    ms = float(np.median(regions))
    barrier()
    # end to end through the C ABI from pinned host buffers: upload the state, K steps,
    # download the state and the ledger
    mh, ml, v1, v2 = R.state()
    t0c, _, s0 = R.clock()
    led = R.ledger()
    cum = np.cumsum(R.hydrograph()) * sc.sample_dt          # the samples recorded up to t0c
    host = [torch.from_numpy(a).pin_memory() for a in (mh, ml, v1, v2)]
    outs = [torch.empty_like(h).pin_memory() for h in host]
    barrier()
    w0 = time.perf_counter()
    A.asx_set_state(R.handle, *[h.data_ptr() for h in host], A.ASX_PTR_HOST, t0c, s0, led, cum)
    R.step(args.steps)
    A.asx_get_state(R.handle, *[o.data_ptr() for o in outs], A.ASX_PTR_HOST)
    led2 = R.ledger()
    barrier()
    e2e_s = time.perf_counter() - w0
    R.close()
    if ws > 1:
        ms, e2e_s = max_over_ranks([ms, e2e_s], "cuda")
    if rank != 0:
        return None
    ms_step = ms / args.steps
    value = job_rate(ws, n, args.steps, ms / 1e3)
    peak, peak_kind = _peaks()
    achieved = BYTES_PER_CELL * n / (ms_step / 1e3) / 1e9
    traffic = _read_traffic(n) if os.environ.get("ASX_STEP_KERNEL", "strip") == "strip" else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded fBm catchment, carved channels, land-cover classes)",
        "config": dict(_workload_config(sc, args.steps, args.t_warm), warm_steps=warm_steps,
                       step_kernel=os.environ.get("ASX_STEP_KERNEL", "strip"),
                       tile_rows=int(os.environ.get("ASX_TILE_ROWS", "32"))),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_kind} copy bandwidth",
                     "note": "32 B algorithmic per cell-update / (step time incl. launch gap); "
                             "traffic: ncu DRAM bytes of one launch on this window, counted over consecutive "
                             "launches without cache control (write-back included)"},
        "e2e": {"value": job_rate(ws, n, args.steps, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": 16 * n / args.steps, "d2h_bytes_per_step": 16 * n / args.steps},
        "gpu_launches": len(regions) * (args.steps + 1),
        "timed_regions": {"count": len(regions), "steps_each": args.steps, "ms_median": ms,
                          "ms_min": float(min(regions)), "ms_max": float(max(regions)),
                          "note": "value and ms_per_step from the median region"},
        "clocks": clk.summary(),
        "mass_defect_rel": led2.defect_rel,
    }
    if args.full_run:
        out["full_run"] = run_full_storm(sc, local, stream)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(sc, budget_s=args.cpu_budget)
    if args.ens_scenarios > 0:
        out["ensemble"] = run_ensemble(args, stream)
    if args.sur_train > 0:
        out["surrogate"] = run_surrogate(args)
    if args.cal:
        out["calibration"] = run_calibration(args)
    return out


TRAFFIC_SOURCES = ("paper_2406_14933_gb300/csrc/step_strip.cu",
                   "paper_2406_14933_gb300/csrc/strip_tile.cuh",
                   "paper_2406_14933_gb300/csrc/device_common.cuh",
                   "paper_2406_14933_gb300/csrc/asx_internal.cuh")


def _read_traffic(n_cells):
    """DRAM bytes (read + write) of one step launch, from the committed ncu summary of a
    smaller window of the same workload, scaled by cells; None when the kernel sources
    have changed since those counters were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "step_strip_kernel__traffic.txt")
    try:
        rec = {}
        with open(path) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                k, v = line.split()
                rec[k] = v
        h = hashlib.sha256()
        for src in TRAFFIC_SOURCES:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != rec["kernel_sources_sha256"]:
            return None
        per_cell = (float(rec["dram_bytes_read"]) + float(rec["dram_bytes_write"])) / float(rec["cells"])
        return per_cell * n_cells
    except Exception:
        return None


def _film_state(sc, depth=0.005):
    h = np.full((sc.rows, sc.cols), depth, np.float32)
    return h, np.zeros_like(h), np.zeros_like(h)


def cpu_baseline(sc, budget_s=15.0, crop=REF_CROP):
    """The FP64 oracle (its OpenMP build, on every core this process may use) on a crop of
    the same raster (a 5 mm film at t = 45 min), timed for about budget_s seconds."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    r0 = (sc.rows - crop) // 2
    c0 = (sc.cols - crop) // 2
    sl = (slice(r0, r0 + crop), slice(c0, c0 + crop))
    cls = sc.cls[sl]
    p = oracle.Problem(crop, crop, sc.l, sc.z[sl], sc.class_theta[cls], sc.class_alpha_s[cls],
                       sc.class_alpha_p[cls], bc=(0, 0, 1, 0), g=sc.g, cfl=sc.cfl,
                       dt_max=sc.dt_max, rain_t=sc.rain_t, rain_r=sc.rain_r, threads=threads)
    h, v1, v2 = _film_state(sc)
    m = p.mass(h[sl])
    a, b = v1[sl].ravel().astype(np.float64), v2[sl].ravel().astype(np.float64)
    t = T_WARM
    steps = 0
    w0 = time.perf_counter()
    while True:
        res = p.run(m, a, b, t, 1e9, max_steps=5)
        m, a, b, t = res["m"], res["v1"], res["v2"], res["t"]
        steps += 5
        if time.perf_counter() - w0 > budget_s:
            break
    el = time.perf_counter() - w0
    return {"value": crop * crop * steps / el, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{steps} oracle steps of a {crop}x{crop} crop of the catchment "
                      f"(5 mm film from t={T_WARM:.0f} s), {el:.1f} s, OpenMP build on {threads} threads",
            "host": host_info()}


def host_info():
    """CPU model and the cores this process may run on."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return {"cpu": model, "machine": platform.machine(), "cores_available": n}


def rain_integral(rain_t, rain_r, t_end):
    """Integral of the piecewise-linear rain rate over [0, t_end] (zero outside the table),
    segment by segment: the exact volume per unit area that the right-endpoint rain of
    each step approximates to O(dt)."""
    total = 0.0
    for k in range(len(rain_t) - 1):
        t0, t1, r0, r1 = rain_t[k], rain_t[k + 1], rain_r[k], rain_r[k + 1]
        a, b = max(t0, 0.0), min(t1, t_end)
        if b <= a or t1 <= t0:
            continue
        ra = r0 + (r1 - r0) * (a - t0) / (t1 - t0)
        rb = r0 + (r1 - r0) * (b - t0) / (t1 - t0)
        total += 0.5 * (b - a) * (ra + rb)
    return total


def run_full_storm(sc, device, stream):
    """The catchment from its dry start through the whole storm to t_end (2 h), one raster,
    CUDA events around the run (host launches and clock reads included): steps, seconds,
    mean cell-updates/s, the water budget and the outlet hydrograph's peak."""
    import numpy as np
    import torch
    from paper_2406_14933_gb300.raster import Raster
    R = Raster(sc, device=device, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    R.run_until(sc.t_end)
    e1.record(stream)
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    t, _, steps = R.clock()
    led = R.ledger()
    q = R.hydrograph()
    R.close()
    k = int(np.argmax(q)) if len(q) else 0
    sigma = 1.5 * math.sqrt(3.0) * sc.l * sc.l
    rain_exact = sc.n * sigma * rain_integral(list(map(float, sc.rain_t)), list(map(float, sc.rain_r)), sc.t_end)
    return {"workload": f"carved catchment {sc.rows}x{sc.cols}, dry start to t = {sc.t_end:.0f} s",
            "t_end": t, "steps": steps, "seconds": s, "cell_updates_per_s": sc.n * steps / s,
            "mean_dt_s": t / max(steps, 1), "rain_m3": led.rain_in,
            "rain_exact_m3": rain_exact, "rain_quadrature_rel": (led.rain_in - rain_exact) / rain_exact,
            "outflow_m3": led.outflow,
            "storage_m3": led.storage - led.storage0, "clamped_m3": led.clamped,
            "mass_defect_rel": led.defect_rel, "hydrograph_samples": len(q),
            "peak_discharge_m3_s": float(q[k]) if len(q) else None,
            "peak_interval_s": [k * sc.sample_dt, (k + 1) * sc.sample_dt] if len(q) else None}


def run_ensemble(args, stream):
    """Batched ensemble of uneven hillslope scenarios (sides 128-512 log-uniform, each run
    to its t_end) in one persistent launch, against one launch per scenario per step (the
    single-raster path run scenario by scenario) on a seeded subsample of the scenarios,
    scaled to the whole ensemble by cell-updates."""
    import torch
    from paper_2406_14933_gb300 import inputs
    from paper_2406_14933_gb300.ensemble import Ensemble
    from paper_2406_14933_gb300.raster import Raster
    n = args.ens_scenarios
    scs = [inputs.ensemble_member(s, t_end=args.ens_t_end) for s in range(n)]
    cells = sum(sc.n for sc in scs)
    E = Ensemble(scs, stream=stream.cuda_stream)
    forced = tuple(int(x) for x in args.ens_tuning.split(",")) if args.ens_tuning else None
    E.run(forced)                             # untimed: each scenario's step count
    if forced:
        from paper_2406_14933_gb300 import asx as A
        tuning = A.asx_ensemble_tuning(*forced)
    else:
        tuning = E.autotune(max_steps=200)    # cut in proportion to those step counts
    E.run(tuning)                             # warm-up (graph capture of the tuned shape)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    E.run(tuning)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ens = e0.elapsed_time(e1) / 1e3
    steps = [E.clock(i)[1] for i in range(n)]
    cell_steps = sum(st * sc.n for st, sc in zip(steps, scs))
    E.close()
    # one launch per scenario per step, on a seeded subsample
    sub = sorted(np.random.default_rng(4242).choice(n, min(n, args.ens_baseline), replace=False).tolist())
    rasters = [Raster(scs[i], stream=stream.cuda_stream) for i in sub]
    torch.cuda.synchronize()
    e0.record(stream)
    for R, i in zip(rasters, sub):
        R.run_until(scs[i].t_end)
    e1.record(stream)
    torch.cuda.synchronize()
    t_sub = e0.elapsed_time(e1) / 1e3
    sub_cell_steps = sum(R.clock()[2] * scs[i].n for R, i in zip(rasters, sub))
    for R in rasters:
        R.close()
    t_one = t_sub * cell_steps / sub_cell_steps
    peak, kind = _peaks()
    achieved = BYTES_PER_CELL * cell_steps / t_ens / 1e9
    return {"workload": f"{n} hillslope scenarios, sides 128-512 log-uniform, {cells} cells, "
                        f"{args.ens_t_end:.0f} s simulated each (rain 10-150 mm/h for 20-60 min, then the recession)",
            "scenarios_per_s": n / t_ens, "cell_updates_per_s": cell_steps / t_ens,
            "steps_total": int(sum(steps)), "seconds": t_ens,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": f"{kind} copy bandwidth",
                         "note": "32 B algorithmic per cell-update / ensemble wall time"},
            "tuning": {"cluster": tuning.cluster, "threads": tuning.threads,
                       "cells_per_thread": tuning.cells_per_thread, "tile_rows": tuning.tile_rows,
                       "split": tuning.split},
            "one_launch_per_scenario": {"scenarios_per_s": n / t_one, "seconds_estimate": t_one,
                                        "timed_subsample": sub, "subsample_seconds": t_sub,
                                        "scaling": "subsample time x (ensemble cell-updates / subsample cell-updates)"},
            "speedup": t_one / t_ens}


def run_calibration(args):
    """The flume study of Sec. 4.3 on the batched ensemble: the 21 x 26 sensitivity grid
    (546 flume runs to a steady state in one ensemble) and the pattern search recovering
    known friction coefficients from solver-made gauges (six experiments per point)."""
    import time
    from paper_2406_14933_gb300 import calibration as C
    from paper_2406_14933_gb300 import inputs
    study = C.FlumeStudy()
    r = C.sensitivity_grid(study, 1, 0.015)
    sc = study.scenario(0.00709, 73.39, 1, 0.015)
    grid = {"workload": f"flume 18 m x 1 m, {sc.rows}x{sc.cols} hex (l = {sc.l} m), 15 l/s, vegetation on "
                        f"x >= 9 m, {study.t_end:.0f} s to a steady state; 21 x 26 (alpha_s, alpha_p) grid",
            "scenarios": study.runs, "solve_seconds": study.solve_seconds,
            "scenarios_per_s": study.runs / study.solve_seconds,
            "cell_updates_per_s": study.cell_updates / study.solve_seconds,
            "end_to_end_seconds": study.seconds, "tune_seconds": study.tune_seconds,
            "tuning": list(study.tuning), "delta_s": r["delta_s"], "delta_p": r["delta_p"],
            "h_bar_range": [float(r["h_bar"].min()), float(r["h_bar"].max())]}
    sweep_study = C.FlumeStudy(tuning=study.tuning)
    envs = [dict(q=0.007), dict(q=0.015), dict(q=0.021), dict(q=0.015, theta_v=0.98),
            dict(q=0.015, slope=0.5e-3), dict(q=0.015, slope=3.0e-3)]
    sw = C.sensitivity_sweep(sweep_study, envs)
    grid["environments"] = {
        "runs": sweep_study.runs, "solve_seconds": sweep_study.solve_seconds,
        "scenarios_per_s": sweep_study.runs / sweep_study.solve_seconds,
        "end_to_end_seconds": sweep_study.seconds,
        "delta": [{"q": e["env"]["q"], "theta_v": e["env"].get("theta_v", inputs.FLUME["theta_v"]),
                   "slope": e["env"].get("slope", inputs.FLUME["slope"]), "delta_s": e["delta_s"],
                   "delta_p": e["delta_p"]} for e in sw]}
    cal_study = C.FlumeStudy(l=0.2, t_end=400.0)
    truth = (0.00709, 73.39)
    h_exp = C.synthetic_gauges(cal_study, *truth)
    s_cases = cal_study.solve_seconds
    surf = C.chi_surfaces(cal_study, h_exp)
    cases = {"solve_seconds": cal_study.solve_seconds - s_cases, "runs": 546 * len(cal_study.experiments)}
    for name, c in surf["cases"].items():
        cases[name] = {"argmin": list(c["argmin"]), "min_chi_m": c["min"],
                       "low_points": int((c["chi"] <= 2.0 * c["min"] + 1e-4).sum())}
    t_gauges, s_gauges, r_gauges = cal_study.seconds, cal_study.solve_seconds, cal_study.runs
    res = C.calibrate(cal_study, h_exp, tol=2e-3)
    search = {"workload": "six experiments (2 vegetation layouts x 3 discharges), 17 gauges each, l = 0.2 m, "
                          "400 s per run; gauges made by the solver at alpha = (0.00709, 73.39)",
              "found": [float(v) for v in res.x], "truth": list(truth), "chi_m": res.f,
              "points": res.evals, "batches": res.batches, "runs": cal_study.runs - r_gauges,
              "solve_seconds": cal_study.solve_seconds - s_gauges, "end_to_end_seconds": cal_study.seconds - t_gauges}
    search["chi_grid_cases"] = cases
    out = {"sensitivity": grid, "estimation": search}
    if not args.no_cpu_baseline:
        import oracle as orc
        p = orc.from_scenario(sc)
        t0 = time.perf_counter()
        p.run(p.mass(sc.h0), sc.v1_0.ravel().astype(float), sc.v2_0.ravel().astype(float), 0.0, sc.t_end)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"kind": "oracle", "cores": 1, "sample": "one flume run of the grid",
                               "scenarios_per_s": 1.0 / dt, "grid_seconds_estimate": dt * study.runs}
    return out


MLP_FLOP_PER_QUERY = 2 * (36 * 256 + 256 * 256 + 256 * 256 + 256 * 128)   # algorithmic (unpadded)
# one training sample: the forward pass, the weight gradients (as many FLOP) and the input
# gradients of layers 2-4 (layer 1's input needs none)
MLP_FLOP_PER_TRAIN_SAMPLE = 2 * MLP_FLOP_PER_QUERY + 2 * (256 * 256 + 256 * 256 + 256 * 128)


def run_surrogate(args):
    """The learned surrogate: training runs from the ensemble solver, training on the GPU,
    held-out error, the inference kernels on 65,536 queries (tensor roofline), and serving
    with a 1 % solver check against the solver alone."""
    import torch
    from paper_2406_14933_gb300 import asx as A
    from paper_2406_14933_gb300 import surrogate as S
    _, peak_kind = _peaks()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        bf16_peak = 1900.0
    rep, model = S.pipeline(n=args.sur_n, l=args.sur_l, n_train=args.sur_train, n_held=args.sur_held,
                            n_queries=args.sur_queries, epochs=args.sur_epochs,
                            workers=min(8, os.cpu_count() or 1), chunk=4096)
    # the forward kernels alone: 65,536 device-resident queries, CUDA events
    Xq, _ = S.query_features(S.QUERY_SEED0, args.sur_queries, args.sur_n, args.sur_l)
    X = torch.as_tensor(Xq, device="cuda")
    Y = torch.empty((X.shape[0], S.N_HYDRO_OUT), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        A.asx_mlp_forward(model.handle, X.shape[0], X.data_ptr(), Y.data_ptr(), A.ASX_PTR_DEVICE)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        A.asx_mlp_forward(model.handle, X.shape[0], X.data_ptr(), Y.data_ptr(), A.ASX_PTR_DEVICE)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    model.close()
    tflops = MLP_FLOP_PER_QUERY * X.shape[0] / (ms / 1e3) / 1e12
    full = args.sur_n == 256 and args.sur_l == 2.0 and args.sur_train >= 20000
    rep["workload"] = (rep["workload"] + (", the surrogate configuration's size" if full else
                       f"; proxy, not the 256x256 / 20,000-run configuration: {args.sur_n}x{args.sur_n} members at "
                       f"l = {args.sur_l:g} m (the same 512 m hillslope), {args.sur_train} training runs"))
    tr = rep["train"]
    train_tflops = MLP_FLOP_PER_TRAIN_SAMPLE * tr["batch"] * tr["steps"] / tr["fit_seconds"] / 1e12
    rep["training"] = {"steps": tr["steps"], "batch": tr["batch"], "seconds": tr["fit_seconds"],
                       "ms_per_step": tr["fit_seconds"] * 1e3 / max(tr["steps"], 1),
                       "roofline": {"bound": "tensor", "achieved": train_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                                    "frac": train_tflops / bf16_peak, "traffic": None,
                                    "note": f"{MLP_FLOP_PER_TRAIN_SAMPLE} algorithmic FLOP per sample and step "
                                            "(forward, weight and input gradients) over the whole fit: host-driven "
                                            "steps of small batches, every kernel, minibatch gathers and launches"}}
    rep["inference"] = {"queries": int(X.shape[0]), "ms": ms, "queries_per_s": X.shape[0] / (ms / 1e3),
                        "roofline": {"bound": "tensor", "achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                                     "frac": tflops / bf16_peak, "traffic": None,
                                     "peak_source": "measured bf16 (burst)" if peak_kind == "measured" else "fallback",
                                     "note": f"{MLP_FLOP_PER_QUERY} algorithmic FLOP per query "
                                             "(the kernel also multiplies layer 1's zero padding to K=64)"}}
    return rep


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return None
    from paper_2406_14933_gb300 import inputs
    sc = inputs.carved_catchment()
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    crop = REF_CROP
    r0, c0 = (sc.rows - crop) // 2, (sc.cols - crop) // 2
    sl = (slice(r0, r0 + crop), slice(c0, c0 + crop))
    cls = sc.cls[sl]
    p = oracle.Problem(crop, crop, sc.l, sc.z[sl], sc.class_theta[cls], sc.class_alpha_s[cls],
                       sc.class_alpha_p[cls], bc=(0, 0, 1, 0), g=sc.g, cfl=sc.cfl,
                       dt_max=sc.dt_max, rain_t=sc.rain_t, rain_r=sc.rain_r, threads=threads)
    h, v1, v2 = _film_state(sc)
    m = p.mass(h[sl])
    a, b = v1[sl].ravel().astype(np.float64), v2[sl].ravel().astype(np.float64)
    t = T_WARM
    for _ in range(args.warmup):
        res = p.run(m, a, b, t, 1e9, max_steps=1)
        m, a, b, t = res["m"], res["v1"], res["v2"], res["t"]
    w0 = time.perf_counter()
    for _ in range(args.steps):
        res = p.run(m, a, b, t, 1e9, max_steps=1)
        m, a, b, t = res["m"], res["v1"], res["v2"], res["t"]
    el = time.perf_counter() - w0
    value = crop * crop * args.steps / el
    cfg = _workload_config(sc, args.steps)
    cfg["reference_crop"] = f"{crop}x{crop} cells per step"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} oracle steps of a {crop}x{crop} crop "
                                       f"(5 mm film from t={T_WARM:.0f} s), OpenMP build on {threads} threads",
                             "host": host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--min-timed-s", type=float, default=0.5,
                    help="repeat the K-step timed region until this much time is timed [s]")
    ap.add_argument("--max-regions", type=int, default=400)
    ap.add_argument("--rows", type=int, default=4096)
    ap.add_argument("--cols", type=int, default=4096)
    ap.add_argument("--t-warm", type=float, default=T_WARM,
                    help="simulated time before the timed window [s]")
    ap.add_argument("--ens-scenarios", type=int, default=256,
                    help="scenarios of the ensemble section (0 = skip it)")
    ap.add_argument("--ens-t-end", type=float, default=6400.0,
                    help="simulated time of each ensemble scenario [s] (the workload's 6400 s)")
    ap.add_argument("--ens-tuning", default="",
                    help="ensemble launch shape cluster,threads,cells_per_thread,tile_rows (default: autotuned)")
    ap.add_argument("--ens-baseline", type=int, default=8,
                    help="scenarios timed one launch per scenario per step (scaled to all by cell-updates)")
    ap.add_argument("--sur-train", type=int, default=16384,
                    help="solver runs the surrogate trains on (0 = skip the surrogate section)")
    ap.add_argument("--sur-held", type=int, default=1000)
    ap.add_argument("--sur-queries", type=int, default=65536)
    ap.add_argument("--sur-epochs", type=int, default=100)
    ap.add_argument("--sur-n", type=int, default=64, help="surrogate members' raster side [cells]")
    ap.add_argument("--sur-l", type=float, default=8.0, help="surrogate members' hexagon edge [m]")
    ap.add_argument("--full-run", type=int, default=1, help="the catchment's whole 2 h storm from a dry start (0: skip)")
    ap.add_argument("--cal", type=int, default=1, help="flume sensitivity grid and coefficient estimation (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    out = run_reference(args) if args.impl == "reference" else run_cuda(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
