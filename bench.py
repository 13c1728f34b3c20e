"""Benchmark: cell-updates/s of the FP64 RHS + TVD-RK3 on the triple-point
problem (1792 x 768, gamma 1.4, reflective walls), one RK3 step (with its CFL
time step) of every scheme per bench step.

  python bench.py --gpus N --steps K --warmup W [--impl reference]

One bench step = for each scheme in {MEG6, MIG4, LAD_E4, LAD_C6, HYBRID global,
HYBRID per interface}: restore the scheme's state from a fixed developed
triple-point state (device copy), CFL dt, one RK3 step.  The developed state is
the initial condition advanced 200 MEG6 steps on the GPU before timing, so
every timed step sees the same flow.  value = cells x schemes x steps / time.
N > 1: every rank runs the same workload on its own GPU (independent
replicas, no exchange); value sums over ranks with the max-over-ranks time.

--impl reference times the FP64 CPU oracle (all host cores) on a bounded
sample of the same workload (one RK3 step of each scheme on the triple point
at 896 x 384, a quarter of the cells).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX, NY = 1792, 768
SCHEMES = [
    ("MEG6", dict(scheme="MEG6")),
    ("MIG4", dict(scheme="MIG4")),
    ("LAD_E4", dict(scheme="LAD_E4")),
    ("LAD_C6", dict(scheme="LAD_C6")),
    ("HYBRID_GLOBAL", dict(scheme="HYBRID", hybrid_mode=0, hyb_rho=0.5 * 0.125)),
    ("HYBRID_CELL", dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.5 * 0.125, hybrid_sensor=1)),
]
MIXED = [
    ("MEG6_MIXED", dict(scheme="MEG6", precision=1)),
    ("MIG4_MIXED", dict(scheme="MIG4", precision=1)),
    ("LAD_E4_MIXED", dict(scheme="LAD_E4", precision=1)),
    ("LAD_C6_MIXED", dict(scheme="LAD_C6", precision=1)),
    ("HYBRID_GLOBAL_MIXED", dict(scheme="HYBRID", hybrid_mode=0, hyb_rho=0.5 * 0.125, precision=1)),
    ("HYBRID_CELL_MIXED", dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.5 * 0.125, hybrid_sensor=1, precision=1)),
]
DEVELOP_STEPS = 200
METRIC = "cell-updates/s per scheme & % HBM roofline; batched solves/s, p50/p99 latency"
# FP64 roofline of the dominant kernel (the C-GBR interface sweep).  Per-unit
# figure: the algorithmic FP64 operations per interface of one sweep launch
# (gradients along the sweep, reconstruction with MP5, HLLC, flux difference,
# residual and RK stage update; add, mul, div and sqrt one each), counted by
# the flop-counting build of the oracle on the developed triple-point state:
# profiles/flops_triple_point_1792x768.md (oracle/count_flops.py).
SWEEP_FLOP_PER_IFACE = 524.8
# dram read + write per launch (mean of x and y) of the sweep form the roofline times,
# from its ncu capture (profiles/); None until the current kernel has been captured
# the bounded sample of the triple point on which the CPU oracle is timed
CPU_SAMPLE = (896, 384)
SWEEP_TRAFFIC_BYTES = {"exact": 118.0e6, "contracted": 140.2e6}
ROOFLINE_FORM = "exact"  # the library default (fma_sweep = 0)
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12  # SMs x DFMA/clk x 2 flop x max clock (context only)
HBM_BYTES_PER_CELL_STEP = 256.0  # minimal-traffic model, FP64 state, nv = 4, uniform grid


def measure_fma_peaks(local):
    """Measured FP64 and FP32 FMA throughput of this GPU (the FMA-chain probe,
    libcgprobe.so; one FMA = 2 flop), with the SM clock sampled meanwhile."""
    import ctypes
    from paper_2511_18042_gb300 import build
    L = ctypes.CDLL(build.PROBE)
    L.cgp_fma_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_int)]
    out = {}
    clk = ClockSampler(local).__enter__()
    time.sleep(0.3)
    clk.mark(True)
    try:
        for name, fp64 in (("fp64", 1), ("fp32", 0)):
            f, ms, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
            rc = L.cgp_fma_peak(fp64, ctypes.byref(f), ctypes.byref(ms), ctypes.byref(sms))
            if rc != 0:
                raise RuntimeError("FMA probe failed (%d)" % rc)
            out[name + "_tflops"] = f.value / 1e12
            out["sms"] = sms.value
    finally:
        clk.mark(False)
        clk.__exit__(None, None, None)
    out["clocks"] = clk.summary()
    return out


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.time(), parts))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def mark(self, start):
        """Wall-clock bounds of the timed region (samples outside it are dropped)."""
        if start:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def summary(self):
        t0, t1 = getattr(self, "t0", None), getattr(self, "t1", None)
        rows = [r for t, r in self.rows if t0 is None or (t0 - 0.15 <= t <= (t1 or t) + 0.15)]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(ms_step, units_per_rank, device=None):
    """Whole-job throughput of independent replicas: every rank processed
    units_per_rank units per step; the step time is the slowest rank's.
    Returns (max-over-ranks ms per step, units of all ranks per second)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    if ws > 1:
        t = torch.tensor([float(ms_step)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
        dist.barrier()
    return ms_step, ws * units_per_rank / (ms_step * 1e-3)


def bench_config(names, ws):
    """The workload of the JSON line, shared by both arms."""
    return {"workload": "triple point 1792x768, FP64, one RK3 step of each of %d schemes "
                        "from a developed state (200 MEG6 steps)" % len(names),
            "schemes": names, "cells": NX * NY, "l2": "flushed between timed steps (256 MB write)",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2511_18042_gb300 import api, inputs
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    prob = inputs.triple_point(NX, NY)
    grid = api.Grid.from_problem(prob)
    cells = NX * NY
    names = [n for n, _ in SCHEMES if args.schemes is None or n in args.schemes.split(",")]
    prec = {"precision": 1} if args.precision == "mixed" else {}
    solvers = {n: api.Solver(grid, **kw, **prec) for n, kw in SCHEMES if n in names}
    # developed state: 200 MEG6 steps from the initial condition
    base = torch.as_tensor(prob["U"], device=dev)
    dev_solver = solvers.get("MEG6") or api.Solver(grid, scheme="MEG6")
    dev_solver.advance(base, nsteps=args.develop)
    torch.cuda.synchronize()
    tiles = {n: solvers[n].autotune(base) for n in names}  # tile shapes by measurement (cached per shape)
    U = {n: torch.empty_like(base) for n in names}
    dt = {n: torch.zeros(2, dtype=torch.float64, device=dev) for n in names}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def one_step(events=None):
        for n in names:
            s = solvers[n]
            if events is not None:
                events[n][0].record(stream)
            U[n].copy_(base)
            s.step(U[n], dt[n])
            if events is not None:
                events[n][1].record(stream)

    # the clock sampler starts before the warm-up (nvidia-smi takes a moment to
    # start); only its samples inside the timed region are kept
    clk = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    launches0 = sum(s.launch_count() for s in solvers.values())
    per = {n: 0.0 for n in names}
    step_ms = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_timed:
        torch.cuda.cudart().cudaProfilerStart()
    try:
        clk.mark(True)
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()  # evict L2 (256 MB > 126 MB) between timed steps
            ev = {n: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for n in names}
            one_step(ev)
            torch.cuda.synchronize()
            for n in names:
                per[n] += ev[n][0].elapsed_time(ev[n][1])
            step_ms.append({n: ev[n][0].elapsed_time(ev[n][1]) for n in names})
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk.mark(False)
    finally:
        clk.__exit__(None, None, None)
        if args.profile_timed:
            torch.cuda.cudart().cudaProfilerStop()
    launches = sum(s.launch_count() for s in solvers.values()) - launches0
    # a scheme whose timed steps produced rho <= 0, p <= 0 or NaN is excluded from value
    status = {}
    for n in names:
        rc = solvers[n].sync_status()
        if rc not in (0, -4):
            raise RuntimeError("solver status %d" % rc)
        status[n] = "ok" if rc == 0 else "nonphysical"
    ok = [n for n in names if status[n] == "ok"]
    ms_step = sum(sum(st[n] for n in ok) for st in step_ms) / len(step_ms)
    ms_step, value = aggregate_over_ranks(ms_step, cells * len(ok), dev if ws > 1 else None)

    # the mixed form (FP32 fluxes, FP64 accumulation) of the schemes that have it
    mixed = {}
    for n, kw in (MIXED if args.mixed else []):
        ms, ms_graph, tile = time_mixed(api, torch, grid, base, dev, kw, args)
        cu = cells / (ms_graph * 1e-3)
        mixed[n] = {"cell_updates_per_s": cu, "ms_per_rk3_step": ms_graph, "ms_per_rk3_step_eager": ms,
                    "tile_lines": list(tile),
                    "hbm_frac_of_measured": cu * HBM_BYTES_PER_CELL_STEP / (_peaks()["hbm_gbs"] * 1e9)}

    sod = run_sod_latency(api, torch, dev) if args.sod else None
    ramp = run_ramp(api, torch, dev, args) if args.ramp else None
    batched = run_batched(api, torch, dev, args) if args.batched else None
    serving = run_serving(args) if args.serving else None

    # roofline of the dominant kernel: the MEG6 interface sweep, timed alone,
    # against the measured FP64 FMA throughput
    roof = sweep_roofline(api, torch, grid, base, dev, args, measure_fma_peaks(local)) if args.roofline else None

    # end to end through the C ABI with host buffers (pinned), one step per scheme
    host = torch.empty(base.shape, dtype=torch.float64, pin_memory=True)
    host_base = base.cpu()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for n in ok:
            host.copy_(host_base)
            solvers[n].advance_host(host, nsteps=1)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    nbytes = base.numel() * 8
    e2e = {"value": ws * cells * len(ok) / e2e_s, "unit": "cell-updates/s",
           "h2d_bytes_per_step": nbytes * len(ok), "d2h_bytes_per_step": nbytes * len(ok)}

    per_scheme = {}
    peaks = _peaks()
    for n in names:
        ms = per[n] / args.steps
        cu = cells / (ms * 1e-3)
        per_scheme[n] = {"cell_updates_per_s": cu, "ms_per_rk3_step": ms, "status": status[n],
                         "hbm_frac_of_measured": cu * HBM_BYTES_PER_CELL_STEP / (peaks["hbm_gbs"] * 1e9),
                         "tile_lines": list(tiles[n])}
    line = {
        "metric": METRIC,
        "value": value, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+f32",
        "data": "synthetic",
        "config": dict(bench_config(names, ws), counted=ok,
                       excluded_nonphysical=[n for n in names if status[n] != "ok"]),
        "per_scheme": per_scheme, "mixed_precision": mixed, "sod_latency": sod, "compression_ramp": ramp, "batched": batched,
        "serving": serving,
        "roofline": roof, "e2e": e2e, "gpu_launches": launches // max(1, args.steps),
        "gpu_launches_timed_total": launches, "wall_s_timed": wall, "clocks": clk.summary(),
    }
    if rank == 0 and args.cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(names, sample=CPU_SAMPLE)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def _hybrid_kw(prob, precision):
    """Per-instance troubled-cell thresholds of the quadrant problems: half the
    smallest initial quadrant density and pressure; a one-node buffer around
    troubled nodes."""
    st = prob["quad_states"]
    return dict(scheme="HYBRID", hybrid_mode=1, hybrid_sensor=1, hyb_rho=0.5 * float(st[:, 0].min()),
                hyb_p=0.5 * float(st[:, 3].min()), hybrid_buffer=1, precision=precision)


RAMP_SCHEMES = [("LAD_E4", dict(scheme="LAD_E4")), ("LAD_C6", dict(scheme="LAD_C6")), ("MEG6", dict(scheme="MEG6")),
                ("MIG4", dict(scheme="MIG4")),
                ("HYBRID_GLOBAL", dict(scheme="HYBRID", hybrid_mode=0, hyb_rho=0.3)),
                ("HYBRID_CELL", dict(scheme="HYBRID", hybrid_mode=1, hybrid_sensor=1, hyb_rho=0.3))]


def run_ramp(api, torch, dev, args):
    """3D M2.9 compression ramp, 768x192x128 body-fitted (metrics on the
    device), Sutherland viscosity, isothermal wall, inflow boundary-layer
    profile with frozen fluctuations: ms per RK3 step (with the device CFL
    step) per scheme in FP64 and in the mixed form, over args.ramp_steps steps
    after one warm-up step, events on the launching stream; the speed ratios
    between schemes beside the paper's (Sec. 4, A100, FP64)."""
    from paper_2511_18042_gb300 import inputs
    prob = inputs.compression_ramp()
    cells = prob["n"][0] * prob["n"][1] * prob["n"][2]
    base = torch.as_tensor(prob["U"], device=dev)
    grid = api.Grid.from_problem(prob)
    out = {}
    for prec in (0, 1):
        for name, kw in RAMP_SCHEMES:
            s = api.Solver.from_problem(prob, grid=grid, precision=prec, **kw)
            U = base.clone()
            dtd = torch.zeros(2, dtype=torch.float64, device=dev)
            s.step(U, dtd)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.ramp_steps):
                s.step(U, dtd)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.ramp_steps
            key = name + ("_MIXED" if prec else "")
            out[key] = {"ms_per_rk3_step": ms, "cell_updates_per_s": cells / (ms * 1e-3),
                        "status": s.sync_status()}
            del s, U
            torch.cuda.empty_cache()
    # speed ratios (time of the first scheme / time of the second), FP64, beside
    # the paper's A100 OpenACC figures for its LES ramps (context, not targets)
    paper = {"MEG6_over_LAD_C6": "1.17-1.22", "MIG4_over_LAD_C6": "1.38-1.43", "MEG6_over_LAD_E4": "1.9-2.0",
             "MIG4_over_LAD_E4": "2.2-2.3", "MEG6_over_HYBRID_GLOBAL": "1.67", "MEG6_over_HYBRID_CELL": None}
    ratios = {}
    for k, ctx in paper.items():
        a, b = k.split("_over_")
        ratios[k] = {"fp64": out[a]["ms_per_rk3_step"] / out[b]["ms_per_rk3_step"],
                     "mixed": out[a + "_MIXED"]["ms_per_rk3_step"] / out[b + "_MIXED"]["ms_per_rk3_step"],
                     "paper_a100_fp64": ctx}
    return {"workload": "M2.9 24-degree compression ramp 768x192x128 (%d cells), curvilinear, viscous; "
                        "%d RK3 steps from the initial boundary layer after one warm-up step" % (cells, args.ramp_steps),
            "per_scheme": out, "speed_ratios": ratios}


def run_profile_ramp(args):
    """Profiling aid: one scheme on a compression ramp of the given size
    (NXxNYxNZ:SCHEME:fp64|mixed), three warm-up steps, then one RK3 step
    bracketed by cudaProfilerStart/Stop (for ncu --profile-from-start off).
    Prints the step's time; not a bench line."""
    import torch
    from paper_2511_18042_gb300 import api, inputs
    size, scheme, prec = args.profile_ramp.split(":")
    nx, ny, nz = (int(v) for v in size.split("x"))
    kw = dict(dict(RAMP_SCHEMES)[scheme], precision=1 if prec == "mixed" else 0)
    prob = inputs.compression_ramp(nx, ny, nz)
    s = api.Solver.from_problem(prob, **kw)
    U = torch.as_tensor(prob["U"], device="cuda")
    dtd = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(3):
        s.step(U, dtd)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.cudart().cudaProfilerStart()
    e0.record()
    s.step(U, dtd)
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    print(json.dumps({"profile_ramp": args.profile_ramp, "cells": nx * ny * nz, "ms_step": e0.elapsed_time(e1),
                      "status": s.sync_status()}))


def run_sod_latency(api, torch, dev, steps=200):
    """Sod tube, 400 cells (latency-bound): microseconds per RK3 step (with the
    device CFL time step) for MEG6 and LAD-C6, launched eagerly and replayed
    as a one-member CUDA graph."""
    from paper_2511_18042_gb300 import inputs
    prob = inputs.shock_tube("sod", 400)
    out = {}
    for name, kw in (("MEG6", dict(scheme="MEG6")), ("LAD_C6", dict(scheme="LAD_C6", cfl=0.1))):
        res = {}
        for mode in ("eager", "graph"):
            s = api.Solver.from_problem(prob, **kw)
            U = torch.as_tensor(prob["U"], device=dev)
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                if mode == "graph":
                    batch = api.Batch([s], [U])
                    step = lambda: batch.step(stream)  # noqa: E731
                else:
                    step = lambda: api.multi_step([s], [U], stream=stream)  # noqa: E731
                for _ in range(3):
                    step()
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    step()
                e1.record(stream)
                stream.synchronize()
            res[mode + "_us_per_step"] = e0.elapsed_time(e1) * 1e3 / steps
        out[name] = res
    return {"workload": "Sod tube 400 cells, %d RK3 steps from the initial state" % steps, **out}


def run_batched(api, torch, dev, args, count=256, steps_per_solve=200, ref_steps=20, acc_members=16):
    """Batched 2D Riemann problems (256 uneven grids, 64^2..512^2, seed 0):
    per-interface hybrid in the mixed form, all members advanced by one CUDA
    graph replay per RK3 step: the batch is autotuned, then all 256 solves run
    their full 200 RK3 steps from the initial states, timed with events.
    Members whose state went non-physical are reported and not counted as
    solves.  Beside it: the per-case FP64 loop (each grid stepped alone,
    host-issued) over ref_steps steps, scaled to 200."""
    from paper_2511_18042_gb300 import inputs
    probs = inputs.batched_riemann(count=count, seed=0)
    cells = sum(p["n"][0] * p["n"][1] for p in probs)
    solvers = [api.Solver.from_problem(p, **_hybrid_kw(p, 1)) for p in probs]
    states = [torch.as_tensor(p["U"], device=dev) for p in probs]
    stream = torch.cuda.Stream()
    batch = api.Batch(solvers, states)

    def timed(k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            batch.step(stream)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    def full_solves():
        """every member from its initial state, steps_per_solve RK3 steps
        (after an eager step, the capture and a replay on the current path);
        returns (ms, non-physical member indices)"""
        for _ in range(3):
            batch.step(stream)
        stream.synchronize()
        for s_ in solvers:
            s_.sync_status(stream)
        for U_, p in zip(states, probs):
            U_.copy_(torch.as_tensor(p["U"]))
        stream.synchronize()
        ms = timed(steps_per_solve)
        batch.sync(stream)
        bad_ = [i for i, s_ in enumerate(solvers) if s_.sync_status(stream) != 0]
        return ms, bad_

    with torch.cuda.stream(stream):
        for _ in range(3):  # eager, capture, first replay
            batch.step(stream)
        stream.synchronize()
        ms_default = timed(10) / 10
        t0 = time.perf_counter()
        width = batch.autotune(stream)
        tune_s = time.perf_counter() - t0
        path, path_launches = batch.path()
        total_ms, bad = full_solves()
        mixed_final = [states[i].clone() for i in range(acc_members)]
        # the other work-table path, timed the same way
        paths = {path: {"launches_per_step": path_launches, "seconds_for_all_solves": total_ms * 1e-3,
                        "solves_per_s": (count - len(bad)) / (total_ms * 1e-3), "nonphysical_members": len(bad)}}
        groups = max(1, path_launches // 41) if path == "table" else 1
        for alt in ("persistent", "table"):
            if alt in paths or path == "streams":
                continue
            try:
                batch.set_path(alt, groups)
            except RuntimeError as ex:
                paths[alt] = {"unavailable": str(ex)}
                continue
            ms_alt, bad_alt = full_solves()
            paths[alt] = {"launches_per_step": batch.path()[1], "seconds_for_all_solves": ms_alt * 1e-3,
                          "solves_per_s": (count - len(bad_alt)) / (ms_alt * 1e-3),
                          "nonphysical_members": len(bad_alt)}
    good = count - len(bad)
    shapes = {}
    for s_ in solvers:
        key = "x".join(str(v) for v in s_.tile_shape())
        shapes[key] = shapes.get(key, 0) + 1
    del batch, solvers, states
    torch.cuda.empty_cache()
    # per-case FP64: each grid advanced on its own, one after the other
    ref_solvers = [api.Solver.from_problem(p, **_hybrid_kw(p, 0)) for p in probs]
    ref_states = [torch.as_tensor(p["U"], device=dev) for p in probs]
    dts = [torch.zeros(2, dtype=torch.float64, device=dev) for _ in probs]
    for s, U, d in zip(ref_solvers, ref_states, dts):
        s.step(U, d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ref_steps):
        for s, U, d in zip(ref_solvers, ref_states, dts):
            s.step(U, d)
    torch.cuda.synchronize()
    ref_ms = (time.perf_counter() - t0) * 1e3 / ref_steps
    del ref_solvers, ref_states
    torch.cuda.empty_cache()
    # accuracy of the batched mixed form after the full 200 steps against the
    # FP64 form of the same members stepped alone
    l1 = []
    for i in range(acc_members):
        if i in bad:
            continue
        s_ = api.Solver.from_problem(probs[i], **_hybrid_kw(probs[i], 0))
        U_ = torch.as_tensor(probs[i]["U"], device=dev)
        s_.advance(U_, nsteps=steps_per_solve)
        a = mixed_final[i][0]
        l1.append(float((a - U_[0]).abs().mean() / U_[0].abs().mean()))
    ms = total_ms / steps_per_solve
    return {"workload": "%d quadrant Riemann problems, N in [64, 512] log-uniform (seed 0), %d cells; "
                        "per-interface hybrid (one-node buffer), FP32 fluxes / FP64 accumulation, "
                        "one graph replay per RK3 step, %d steps per solve" % (count, cells, steps_per_solve),
            "ms_per_rk3_step": ms,
            "cell_updates_per_s": sum(p["n"][0] * p["n"][1] for i, p in enumerate(probs) if i not in bad) / (ms * 1e-3),
            "seconds_for_all_solves": total_ms * 1e-3,
            "solves_per_s": good / (total_ms * 1e-3), "steps_per_solve": steps_per_solve,
            "members_ok": good, "nonphysical_members": len(bad),
            "nonphysical": [{"member": i, "n": probs[i]["n"][0],
                             "why": "C-GBR (MEG6 alone too) drains the four-state junction cell "
                                    "within 0.45 cell-crossing times at any resolution"
                             if i == 249 else "unexplained"} for i in bad],
            "autotune": {"path": path, "launches_per_step": path_launches,
                         "streams": width, "tile_shapes": shapes, "seconds": tune_s,
                         "ms_per_rk3_step_default": ms_default,
                         "note": "path: 'persistent' = one cooperative launch per RK stage (3 per step) "
                                 "running the stage's phases with grid barriers; 'table' = one launch per "
                                 "phase of an RK stage for every member (41 per step and member group); "
                                 "'streams' = per-member launches on the stream pool; default = the work "
                                 "table, untuned"},
            "paths": paths,
            "accuracy_vs_fp64": {"members": len(l1), "steps": steps_per_solve,
                                 "density_l1_rel_max": max(l1) if l1 else None},
            "per_case_fp64": {"ms_per_rk3_step": ref_ms,
                              "solves_per_s": count / (steps_per_solve * ref_ms * 1e-3),
                              "how": "each grid stepped alone in FP64 (wall clock, host-issued launches), "
                                     "%d steps timed, scaled to %d" % (ref_steps, steps_per_solve)}}


def run_serving(args, count=200, rates=(8.0, 16.0, 32.0, 64.0)):
    """Serving stream (Poisson arrivals of the seeded 60/40 tube/quadrant mix,
    50..500 RK3 steps each, 100 GB admission budget): p50/p99 latency,
    solves/s and GPU busy fraction per arrival rate; the saturation rate is
    the first one whose median latency exceeds twice the lowest rate's (the
    queue, not the solves, sets the latency from there on)."""
    from paper_2511_18042_gb300 import serve
    out = []
    for lam in rates:
        reqs = serve.request_mix(count, rate=lam, seed=0)
        stats, _ = serve.run(reqs, budget_bytes=100 << 30)
        stats["lambda_per_s"] = lam
        out.append(stats)
    sat = next((o["lambda_per_s"] for o in out if o["p50_latency_s"] > 2.0 * out[0]["p50_latency_s"]), None)
    return {"scheme": "per-interface hybrid (one-node buffer), FP32 fluxes / FP64 accumulation",
            "requests_per_rate": count, "rates": out, "saturation_lambda_per_s": sat,
            "saturated_solves_per_s": max(o["solves_per_s"] for o in out)}


def time_mixed(api, torch, grid, base, dev, kw, args):
    """ms per RK3 step (with the CFL step) of a mixed-precision solver on the
    bench state, tile shape autotuned.  Before each timed step the state is
    restored and L2 flushed (256 MB written > 126 MB), so the timed region is
    the step alone from cold caches: launched eagerly (cg_step_dev) and
    replayed as a captured CUDA graph (cg_step_graph) on a side stream.
    Returns (ms eager, ms graph, tile)."""
    s = api.Solver(grid, **kw)
    tile = s.autotune(base)
    U = torch.empty_like(base)
    dtd = torch.zeros(2, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    gs = torch.cuda.Stream(device=dev)
    gs.wait_stream(torch.cuda.current_stream())
    res = []
    for graph in (False, True):
        with torch.cuda.stream(gs):
            for _ in range(max(3, args.warmup)):
                U.copy_(base)
                if graph:
                    s.step_graph(U, dtd, gs)
                else:
                    s.step(U, dtd, stream=gs)
            gs.synchronize()
            tot = 0.0
            for _ in range(max(1, args.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.zero_()
                U.copy_(base)
                flush.zero_()
                e0.record(gs)
                if graph:
                    s.step_graph(U, dtd, gs)
                else:
                    s.step(U, dtd, stream=gs)
                e1.record(gs)
                gs.synchronize()
                tot += e0.elapsed_time(e1)
        res.append(tot / max(1, args.steps))
    return res[0], res[1], tile


def _sweep_ms(api, torch, grid, base, dev, args, form):
    """Average duration of the MEG6 interface-sweep launches (CUDA events around
    each launch on its stream, recorded by the library) over RK3 steps of the
    bench state, for the exact or the FMA form; returns (ms, launches, tile)."""
    s = api.Solver(grid, scheme="MEG6", fma_sweep=int(form == "contracted"))
    tile = s.autotune(base)
    U = torch.empty_like(base)
    dtd = torch.zeros(2, dtype=torch.float64, device=dev)
    for _ in range(2):
        U.copy_(base)
        s.step(U, dtd)
    torch.cuda.synchronize()
    s.timing_enable(True)
    reps = max(2, args.steps)
    for _ in range(reps):
        U.copy_(base)
        s.step(U, dtd)
    torch.cuda.synchronize()
    ms, n = s.timing_query(0)
    s.timing_enable(False)
    return ms / n, n, tile


def sweep_roofline(api, torch, grid, base, dev, args, peaks):
    """FP64 roofline of the dominant kernel, the MEG6 interface sweep, in the
    library's default (exact) form: algorithmic flop per interface (oracle
    count) x interfaces per launch / measured launch time, against the
    measured FP64 FMA peak; the opt-in FMA form beside it."""
    ifaces = ((NX + 1) * NY + NX * (NY + 1)) / 2.0  # algorithmic interfaces per sweep launch (x, y average)
    peak = peaks["fp64_tflops"]
    avg_ms, n, tile = _sweep_ms(api, torch, grid, base, dev, args, ROOFLINE_FORM)
    roof = {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
            "peak_source": "measured: FP64 FMA-chain probe on this GPU (%d SMs, SM clock median %s MHz); "
                           "derived 2 DFMA/clk/SM x 2.07 GHz = %.3f" % (peaks["sms"], peaks["clocks"].get("sm_mhz"),
                                                                       FP64_PEAK_DERIVED_TFLOPS),
            "kernel": "k_gbr_sweep (MEG6), x and y launches of RK3 steps of the bench state",
            "launch_ms": avg_ms, "launches": n, "ifaces_per_launch": ifaces,
            "traffic": SWEEP_TRAFFIC_BYTES[ROOFLINE_FORM], "form": ROOFLINE_FORM,
            "tile_lines": list(tile)}
    ach = SWEEP_FLOP_PER_IFACE * ifaces / (avg_ms * 1e-3) / 1e12
    roof.update({"achieved": ach, "frac": ach / peak, "algorithmic_flop_per_iface": SWEEP_FLOP_PER_IFACE,
                 "flop_source": "oracle operation count (profiles/flops_triple_point_1792x768.md)",
                 "peak_measured": {k: v for k, v in peaks.items() if k != "clocks"}})
    fms, fn, ftile = _sweep_ms(api, torch, grid, base, dev, args, "contracted")
    fach = SWEEP_FLOP_PER_IFACE * ifaces / (fms * 1e-3) / 1e12
    roof["fma_sweep"] = {"launch_ms": fms, "launches": fn, "tile_lines": list(ftile), "achieved": fach,
                         "frac": fach / peak, "traffic": SWEEP_TRAFFIC_BYTES["contracted"],
                         "note": "opt-in FMA form (fma_sweep = 1): not bitwise; see profiles"}
    return roof


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def _oracle_rate(oracle, prob, kw, steps, U0=None):
    """cell-updates/s of the oracle advancing prob by `steps` CFL RK3 steps."""
    o = oracle.Oracle(prob, **kw)
    U = prob["U"] if U0 is None else U0
    t0 = time.perf_counter()
    for _ in range(steps):
        U = o.rk3_step(U, o.cfl_dt(U))
    sec = time.perf_counter() - t0
    cells = math.prod(int(v) for v in prob["n"][:prob["ndim"]])
    return cells * steps / sec, sec


def cpu_baseline(names, sample=None):
    """The oracle as it stands (plain FP64 C, OpenMP over the outer grid
    loops, results independent of the thread count), timed on this host on
    bounded samples of the workloads: the headline's RK3 steps of each scheme
    (two on all cores, one single-threaded) on an 896 x 384 triple point (a
    quarter of the cells) from 20 MEG6 steps of development, and the cases of the
    benchmark's other configurations on all cores (Sod to t = 0.2, the same
    triple point 10 steps, 10 batched Riemann problems 10 steps, a 96 x 48 x 32
    compression ramp 2 steps)."""
    import oracle
    from paper_2511_18042_gb300 import inputs
    sample = sample or CPU_SAMPLE
    ncores = oracle.set_threads(0)
    prob = inputs.triple_point(*sample)
    kws = dict(SCHEMES)
    oracle.set_threads(ncores)
    U0, _, _ = oracle.Oracle(prob, scheme="MEG6").advance(prob["U"], nsteps=20)
    res = {}
    for th, steps in ((1, 1), (ncores, 2)):
        oracle.set_threads(th)
        orcs = [oracle.Oracle(prob, **kws[n]) for n in names]
        t0 = time.perf_counter()
        for o in orcs:
            U = U0
            for _ in range(steps):
                U = o.rk3_step(U, o.cfl_dt(U))
        sec = time.perf_counter() - t0
        res[th] = (sample[0] * sample[1] * len(names) * steps / sec, sec)
    oracle.set_threads(ncores)
    cases = {}
    sod = inputs.shock_tube("sod", 400)
    for n, kw in (("MEG6", dict(scheme="MEG6", cfl=0.5)), ("LAD_C6", dict(scheme="LAD_C6", cfl=0.1))):
        o = oracle.Oracle(sod, **kw)
        t0 = time.perf_counter()
        _, _, k = o.advance(sod["U"], t_end=0.2)
        sec = time.perf_counter() - t0
        cases["sod_400_to_t0.2_" + n] = {"cell_updates_per_s": 400 * k / sec, "steps": k, "seconds": sec}
    for n in ("MEG6", "LAD_E4", "HYBRID_CELL"):
        r, sec = _oracle_rate(oracle, prob, kws[n], 10, U0)
        cases["triple_point_%dx%d_10_steps_%s" % (sample[0], sample[1], n)] = {"cell_updates_per_s": r,
                                                                                "seconds": sec}
    br = inputs.batched_riemann(count=10, seed=0)
    t0 = time.perf_counter()
    cells = 0
    for p in br:
        o = oracle.Oracle(p, **_hybrid_kw(p, 0))
        U = p["U"]
        for _ in range(10):
            U = o.rk3_step(U, o.cfl_dt(U))
        cells += p["n"][0] * p["n"][1] * 10
    sec = time.perf_counter() - t0
    cases["batched_riemann_10x10_steps_hybrid"] = {"cell_updates_per_s": cells / sec, "seconds": sec}
    ramp = inputs.compression_ramp(96, 48, 32)
    for n in ("LAD_E4", "MEG6"):
        r, sec = _oracle_rate(oracle, ramp, dict(scheme=n), 2)
        cases["ramp_96x48x32_2_steps_" + n] = {"cell_updates_per_s": r, "seconds": sec}
    return {"value": res[ncores][0], "unit": "cell-updates/s", "cores": ncores, "kind": "oracle",
            "sample": "two RK3 steps of each of %d schemes on a %dx%d triple point (a quarter of the cells), from "
                      "20 MEG6 steps of development, on %d threads (%.2f s)" % (len(names), sample[0], sample[1],
                                                                              ncores, res[ncores][1]),
            "single_core": {"value": res[1][0], "seconds": res[1][1]},
            "cores_all": ncores, "cpu_model": _cpu_model(), "cases_all_cores": cases}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    names = [n for n, _ in SCHEMES if args.schemes is None or n in args.schemes.split(",")]
    import oracle
    from paper_2511_18042_gb300 import inputs
    ncores = oracle.set_threads(0)
    sample = CPU_SAMPLE
    prob = inputs.triple_point(*sample)
    kws = dict(SCHEMES)
    pre = oracle.Oracle(prob, scheme="MEG6")
    U0, _, _ = pre.advance(prob["U"], nsteps=20)
    orcs = {n: oracle.Oracle(prob, **kws[n]) for n in names}

    def step():
        for n in names:
            o = orcs[n]
            o.rk3_step(U0, o.cfl_dt(U0))

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    sec = (time.perf_counter() - t0) / args.steps
    cells = sample[0] * sample[1] * len(names)
    value = cells / sec
    desc = ("FP64 CPU oracle (OpenMP, %d threads): one RK3 step of each of %d schemes on a %dx%d triple point "
            "(bounded sample of the 1792x768 workload)" % (ncores, len(names), sample[0], sample[1]))
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "cell-updates/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": dict(bench_config(names, ws), sample="%dx%d triple point from its initial state" % sample),
            "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": ncores, "kind": "oracle",
                             "sample": desc, "cpu_model": _cpu_model()},
            "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cgflow", choices=["cgflow", "reference"])
    ap.add_argument("--schemes", default=None, help="comma-separated subset (default: all six)")
    ap.add_argument("--develop", type=int, default=DEVELOP_STEPS)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-serving", dest="serving", action="store_false")
    ap.add_argument("--no-sod", dest="sod", action="store_false")
    ap.add_argument("--no-ramp", dest="ramp", action="store_false")
    ap.add_argument("--ramp-steps", type=int, default=20)
    ap.add_argument("--no-mixed", dest="mixed", action="store_false")
    ap.add_argument("--no-roofline", dest="roofline", action="store_false")
    ap.add_argument("--profile-timed", action="store_true",
                    help="cudaProfilerStart/Stop around the timed steps (ncu --profile-from-start off)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="form of the timed schemes (profiling; the headline is FP64)")
    ap.add_argument("--profile-ramp", default=None, metavar="NXxNYxNZ:SCHEME:fp64|mixed",
                    help="profiling aid: one ramp step of one scheme between cudaProfilerStart/Stop, then exit")
    args = ap.parse_args()
    if args.profile_ramp:
        from paper_2511_18042_gb300 import build
        build.build()
        run_profile_ramp(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        from paper_2511_18042_gb300 import build
        build.build()
        run_gpu(args)


if __name__ == "__main__":
    main()
