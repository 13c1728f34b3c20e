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
from collections import deque
from dataclasses import dataclass

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
    status: str = None
    host: object = None


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
    """Per-interface hybrid with thresholds at half the smallest initial
    density / pressure and a one-node buffer around troubled nodes (the
    random quadrant states hold vortex sheets that LAD-E4 alone cannot carry)."""
    if prob["ndim"] == 1:
        rmin = min(prob["WL"][0], prob["WR"][0])
        pmin = min(prob["WL"][2], prob["WR"][2])
    else:
        st = prob["quad_states"]
        rmin, pmin = float(st[:, 0].min()), float(st[:, 3].min())
    return dict(scheme="HYBRID", hybrid_mode=1, hybrid_sensor=1, hyb_rho=0.5 * rmin, hyb_p=0.5 * pmin,
                hybrid_buffer=1, precision=precision, cfl=0.2)


def state_bytes(prob):
    nv = prob["ndim"] + 2
    return 8 * nv * int(np.prod(prob["n"][:prob["ndim"]]))


def _shape_key(prob, precision):
    return (prob["ndim"], tuple(prob["n"][:prob["ndim"]]), precision)


class _Tick:
    """One enqueued tick: its timing events and the requests whose results
    were copied to the host at its end."""
    __slots__ = ("start", "end", "finished")

    def __init__(self, start, end, finished):
        self.start, self.end, self.finished = start, end, finished


def run(requests, budget_bytes=100 << 30, precision=1, device="cuda", max_active=None, depth=2):
    """Serve the requests; returns (stats dict, finished requests).

    Admission: in arrival order, while the device bytes of the admitted
    requests (their state plus the solver's scratch as the library reports it,
    cg_solver_device_bytes; measured once per grid shape) fit the budget.
    Every tick advances each admitted request by one RK3 step (cg_multi_step
    on the serving stream).  The host does not wait for a tick before
    enqueueing the next: up to `depth` ticks are in flight.  A request that
    takes its last step leaves the batch at once; its state is copied to a
    pinned host buffer behind that tick and it is retired (result, status,
    latency, memory released) when the tick's end event has completed.
    status: "ok", or "nonphysical" when the library's sticky flag reports
    rho <= 0, p <= 0 or NaN in any of its steps; solves/s and the latencies
    count "ok" requests only."""
    dev = torch.device(device)
    pending = sorted(requests, key=lambda r: r.arrival)
    active = []
    used = 0
    sizes = {}
    stream = torch.cuda.Stream(dev)
    side = torch.cuda.Stream(dev)  # status reads: never waits for the serving stream
    inflight = deque()
    done = []
    ticks = 0
    gpu_ms = 0.0
    t0 = time.perf_counter()

    def retire(tk):
        nonlocal used, gpu_ms
        tk.end.synchronize()
        gpu_ms += tk.start.elapsed_time(tk.end)
        t_done = time.perf_counter() - t0
        for r in tk.finished:
            r.status = "ok" if r.solver.sync_status(side) == 0 else "nonphysical"
            r.result = r.host.numpy()
            r.done_at = t_done
            used -= r.bytes
            r.solver = r.state = r.host = None
            done.append(r)

    while pending or active or inflight:
        while inflight and (len(inflight) >= depth or inflight[0].end.query()):
            retire(inflight.popleft())
        now = time.perf_counter() - t0
        # admit in arrival order while the budget allows
        while pending and pending[0].arrival <= now:
            r = pending[0]
            if max_active and len(active) >= max_active:
                break
            key = _shape_key(r.prob, precision)
            solver = None
            if key not in sizes:  # first request of this shape: size it by its solver
                solver = api.Solver.from_problem(r.prob, **solver_kwargs(r.prob, precision))
                sizes[key] = solver.device_bytes() + state_bytes(r.prob)
            need = sizes[key]
            if used + need > budget_bytes:
                break
            pending.pop(0)
            r.solver = solver or api.Solver.from_problem(r.prob, **solver_kwargs(r.prob, precision))
            with torch.cuda.stream(stream):
                r.state = torch.as_tensor(r.prob["U"]).to(dev)
            r.host = torch.empty(r.state.shape, dtype=torch.float64, pin_memory=True)
            r.left = r.steps
            r.bytes = need
            used += need
            active.append(r)
        if not active:
            if inflight:
                retire(inflight.popleft())
                continue
            wait = pending[0].arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(min(wait, 0.05))
            continue
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.multi_step([r.solver for r in active], [r.state for r in active], stream=stream)
        finished, still = [], []
        for r in active:
            r.left -= 1
            if r.left == 0:
                with torch.cuda.stream(stream):
                    r.host.copy_(r.state, non_blocking=True)
                finished.append(r)
            else:
                still.append(r)
        e1.record(stream)
        inflight.append(_Tick(e0, e1, finished))
        ticks += 1
        active = still
    wall = time.perf_counter() - t0
    ok = [r for r in done if r.status == "ok"]
    lat = np.array([r.done_at - r.arrival for r in ok]) if ok else np.zeros(1)
    stats = {"requests": len(done), "ok": len(ok), "nonphysical": len(done) - len(ok),
             "nonphysical_ids": [r.rid for r in done if r.status != "ok"],
             "wall_s": wall, "solves_per_s": len(ok) / wall,
             "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
             "gpu_busy_frac": gpu_ms * 1e-3 / wall, "ticks": ticks,
             "cell_updates": int(sum(r.cells * r.steps for r in ok)),
             "sized_shapes": len(sizes)}
    return stats, done


def run_alone(req, precision=1, device="cuda"):
    """The same request served on its own (for the mix-independence check)."""
    s = api.Solver.from_problem(req.prob, **solver_kwargs(req.prob, precision))
    U = torch.as_tensor(req.prob["U"], device=device)
    s.advance(U, nsteps=req.steps)
    return U.cpu().numpy()
