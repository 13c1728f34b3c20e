"""Continuous-batching request loop for shock-tube and 2D Riemann solves.

Requests arrive over time (Poisson); each asks for a fixed number of RK3 steps
of one problem.  The server keeps every admitted request's state resident on
the GPU, admits waiting requests in arrival order as soon as the memory
budget has room, and advances all admitted requests together, one RK3 step
each per tick, through one native call (cg_multi_step: members run
concurrently on forked streams).  A request that finishes leaves the batch at
once and its result is read back to the host; new requests join at the next
tick.  Latency = result on the host minus arrival.  The scheme is the
per-interface hybrid LAD-GBR in the mixed form (FP32 fluxes, FP64
accumulation) unless told otherwise.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api, inputs


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start
    prob: dict
    steps: int
    kind: str
    cells: int
    done_at: float = None
    result: np.ndarray = None
    state: object = None
    solver: object = None
    left: int = 0
    bytes: int = 0


def request_mix(count, rate, seed=0, tube=(200, 20000), quad=(128, 1024), steps=(50, 500), frac_tube=0.6):
    """Seeded serving mix: Poisson(rate) arrivals; 60 % 1D tubes N ~ logU[200, 20000],
    40 % 2D quadrant problems N ~ logU[128, 1024]; steps ~ U{50..500}."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        if rng.uniform() < frac_tube:
            n = int(round(math.exp(rng.uniform(math.log(tube[0]), math.log(tube[1])))))
            prob = inputs.random_tube(rng, n)
            kind, cells = "tube", n
        else:
            n = int(round(math.exp(rng.uniform(math.log(quad[0]), math.log(quad[1])))))
            prob = inputs.random_quadrants(rng, n)
            kind, cells = "quad", n * n
        nsteps = int(rng.integers(steps[0], steps[1] + 1))
        out.append(Request(i, t, prob, nsteps, kind, cells))
    return out


def solver_kwargs(prob, precision=1):
    """Per-interface hybrid with thresholds at half the smallest initial density / pressure."""
    if prob["ndim"] == 1:
        rmin = min(prob["WL"][0], prob["WR"][0])
        pmin = min(prob["WL"][2], prob["WR"][2])
    else:
        st = prob["quad_states"]
        rmin, pmin = float(st[:, 0].min()), float(st[:, 3].min())
    return dict(scheme="HYBRID", hybrid_mode=1, hybrid_sensor=1, hyb_rho=0.5 * rmin, hyb_p=0.5 * pmin,
                precision=precision, cfl=0.2)


def bytes_estimate(prob):
    """Device bytes a request holds: its state plus the solver's scratch
    (primitives, accumulator, two stage states, sensor, LAD buffers), bounded
    above by 40 FP64 values per cell and variable."""
    nv = prob["ndim"] + 2
    cells = int(np.prod(prob["n"][:prob["ndim"]]))
    return 8 * nv * cells * 40


def run(requests, budget_bytes=100 << 30, precision=1, device="cuda", max_active=None):
    """Serve the requests; returns (stats dict, requests with results)."""
    dev = torch.device(device)
    pending = sorted(requests, key=lambda r: r.arrival)
    active = []
    used = 0
    t0 = time.perf_counter()
    gpu_ms = 0.0
    ticks = 0
    stream = torch.cuda.current_stream(dev)
    done = []
    while pending or active:
        now = time.perf_counter() - t0
        # admit in arrival order while the budget allows
        while pending and pending[0].arrival <= now:
            r = pending[0]
            need = bytes_estimate(r.prob)
            if used + need > budget_bytes or (max_active and len(active) >= max_active):
                break
            pending.pop(0)
            r.solver = api.Solver.from_problem(r.prob, **solver_kwargs(r.prob, precision))
            r.state = torch.as_tensor(r.prob["U"], device=dev)
            r.left = r.steps
            r.bytes = need
            used += need
            active.append(r)
        if not active:
            wait = pending[0].arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.multi_step([r.solver for r in active], [r.state for r in active], stream=stream)
        e1.record(stream)
        e1.synchronize()
        gpu_ms += e0.elapsed_time(e1)
        ticks += 1
        still = []
        for r in active:
            r.left -= 1
            if r.left == 0:
                r.result = r.state.cpu().numpy()
                r.done_at = time.perf_counter() - t0
                used -= r.bytes
                r.solver = None
                r.state = None
                done.append(r)
            else:
                still.append(r)
        active = still
    wall = time.perf_counter() - t0
    lat = np.array([r.done_at - r.arrival for r in done])
    stats = {"requests": len(done), "wall_s": wall, "solves_per_s": len(done) / wall,
             "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
             "gpu_busy_frac": gpu_ms * 1e-3 / wall, "ticks": ticks,
             "cell_updates": int(sum(r.cells * r.steps for r in done))}
    return stats, done


def run_alone(req, precision=1, device="cuda"):
    """The same request served on its own (for the mix-independence check)."""
    s = api.Solver.from_problem(req.prob, **solver_kwargs(req.prob, precision))
    U = torch.as_tensor(req.prob["U"], device=device)
    s.advance(U, nsteps=req.steps)
    return U.cpu().numpy()
