"""Algorithmic FP64 operation counts of the method, per scheme, from the
flop-counting build of the oracle (flopcount.cpp; measurement infrastructure,
like the oracle).

    python oracle/count_flops.py [--nx 1792 --ny 768 --develop 200] [--out FILE]

State: the triple point (Sec. 3.2) developed by `develop` MEG6 steps with the
oracle itself (OpenMP build), the state the benchmark times.  For each scheme,
one CFL time step and one TVD-RK3 step are counted: additions/subtractions,
multiplications, divisions and square roots (one operation each), per step of
the method.  Reported per cell and RK3 step, and, for the C-GBR interface
sweep (gradients along the sweep direction, reconstruction with MP5, HLLC with
its node fluxes, flux difference, residual scaling and the RK stage update:
the work of one fused sweep launch per direction), per interface.
"""
import argparse
import ctypes
import json
import os
import subprocess
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(_HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
_SO = os.path.join(_HERE, "_build", "libcgoracle_count.so")

SCHEMES = [
    ("MEG6", dict(scheme="MEG6")),
    ("MIG4", dict(scheme="MIG4")),
    ("LAD_E4", dict(scheme="LAD_E4")),
    ("LAD_C6", dict(scheme="LAD_C6")),
    ("HYBRID_GLOBAL", dict(scheme="HYBRID", hybrid_mode=0, hyb_rho=0.5 * 0.125)),
    ("HYBRID_CELL", dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.5 * 0.125, hybrid_sensor=1)),
]
# the steps one fused C-GBR interface sweep launch performs
SWEEP_REGIONS = ("grad", "reconstruct", "mp5", "hllc", "node_flux", "flux_diff", "residual", "rk3")


def build(force=False):
    src = [os.path.join(_HERE, f) for f in ("flopcount.cpp", "cg_oracle.c", "cg_oracle.h")]
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(map(os.path.getmtime, src)):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-Wno-unknown-pragmas", "-o", tmp, os.path.join(_HERE, "flopcount.cpp")], cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


class Counter:
    """The counting oracle: same entry points as the oracle library."""

    def __init__(self):
        import oracle
        self.L = ctypes.CDLL(build())
        P = ctypes.POINTER(ctypes.c_double)
        L = self.L
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(oracle.OrcParams), P]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_rhs.argtypes = [ctypes.c_void_p, P, P]
        L.orc_rk3_step.argtypes = [ctypes.c_void_p, P, ctypes.c_double]
        L.orc_cfl_dt.restype = ctypes.c_double
        L.orc_cfl_dt.argtypes = [ctypes.c_void_p, P]
        L.fc_region_name.restype = ctypes.c_char_p
        L.fc_region_name.argtypes = [ctypes.c_int]
        L.fc_region_counts.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)]
        self.oracle = oracle

    def counts(self):
        out = {}
        buf = (ctypes.c_ulonglong * 4)()
        for i in range(self.L.fc_regions()):
            self.L.fc_region_counts(i, buf)
            out[self.L.fc_region_name(i).decode()] = [int(v) for v in buf]
        return out

    def step(self, problem, U, **over):
        """Counts of one CFL time step + one RK3 step from state U; returns
        (counts per region, the new state)."""
        p = self.oracle.make_params(problem, **over)
        ctx = self.L.orc_create(ctypes.byref(p), None)
        U = np.ascontiguousarray(U, dtype=np.float64).copy()
        ptr = U.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self.L.fc_reset()
        dt = self.L.orc_cfl_dt(ctx, ptr)
        self.L.orc_rk3_step(ctx, ptr, dt)
        c = self.counts()
        self.L.orc_destroy(ctx)
        return c, U

    def rhs(self, problem, U, **over):
        p = self.oracle.make_params(problem, **over)
        ctx = self.L.orc_create(ctypes.byref(p), None)
        U = np.ascontiguousarray(U, dtype=np.float64)
        R = np.empty_like(U)
        self.L.fc_reset()
        self.L.orc_rhs(ctx, U.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       R.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        c = self.counts()
        self.L.orc_destroy(ctx)
        return c, R


def total(c, regions=None):
    return sum(sum(v) for k, v in c.items() if regions is None or k in regions)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=1792)
    ap.add_argument("--ny", type=int, default=768)
    ap.add_argument("--develop", type=int, default=200)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import oracle
    from paper_2511_18042_gb300 import inputs
    prob = inputs.triple_point(args.nx, args.ny)
    t0 = time.time()
    threads = oracle.set_threads(0)
    U, _, _ = oracle.Oracle(prob, scheme="MEG6").advance(prob["U"], nsteps=args.develop)
    dev_s = time.time() - t0
    cells = args.nx * args.ny
    ifaces = (args.nx + 1) * args.ny + args.nx * (args.ny + 1)  # per stage, x and y sweeps
    C = Counter()
    rows = {}
    for name, kw in SCHEMES:
        c, _ = C.step(prob, U, **kw)
        rows[name] = c
    res = {"state": "triple point %dx%d after %d MEG6 steps (oracle, %d threads, %.0f s)"
                    % (args.nx, args.ny, args.develop, threads, dev_s),
           "cells": cells, "ifaces_per_stage": ifaces, "schemes": {}}
    for name, c in rows.items():
        per_cell = total(c, [k for k in c if k != "metrics"]) / cells
        ent = {"flop_per_cell_rk3_step": per_cell,
               "by_step_per_cell": {k: sum(v) / cells for k, v in sorted(c.items()) if sum(v)},
               "ops": {k: v for k, v in sorted(c.items()) if sum(v)}}
        if name == "MEG6":
            sw = total(c, SWEEP_REGIONS)
            ent["sweep_flop_per_interface"] = sw / (3 * ifaces)
            kinds = [sum(c[k][i] for k in SWEEP_REGIONS if k in c) for i in range(4)]
            ent["sweep_ops_per_interface"] = dict(zip(("add", "mul", "div", "sqrt"), [v / (3 * ifaces) for v in kinds]))
        res["schemes"][name] = ent
    js = json.dumps(res, indent=1)
    print(js)
    if args.out:
        with open(args.out, "w") as f:
            f.write(_markdown(res, " ".join(["python oracle/count_flops.py"] + sys.argv[1:])))


def _markdown(res, cmd):
    s = ["# Algorithmic FP64 operation counts, triple point", "",
         "Command: `%s`" % cmd, "",
         "Counted by the flop-counting build of the oracle (`oracle/flopcount.cpp`): additions and",
         "subtractions, multiplications, divisions and square roots, one each; comparisons, absolute",
         "values, minima and maxima not counted. One CFL time step plus one TVD-RK3 step per scheme,",
         "on the %s." % res["state"], "",
         "| scheme | flop per cell and RK3 step | largest steps (flop per cell and step) |", "|---|---|---|"]
    for name, e in res["schemes"].items():
        top = sorted(e["by_step_per_cell"].items(), key=lambda t: -t[1])[:5]
        s.append("| %s | %.1f | %s |" % (name, e["flop_per_cell_rk3_step"],
                                          ", ".join("%s %.0f" % (k, v) for k, v in top)))
    m = res["schemes"]["MEG6"]
    o = m["sweep_ops_per_interface"]
    s += ["", "C-GBR (MEG6) interface sweep, per interface (x and y sweeps of the three stages, "
              "%d interfaces per stage): **%.1f flop** (%.1f add, %.1f mul, %.2f div, %.2f sqrt). "
              "Steps counted: %s." % (res["ifaces_per_stage"], m["sweep_flop_per_interface"], o["add"], o["mul"],
                                     o["div"], o["sqrt"], ", ".join(SWEEP_REGIONS)), ""]
    return "\n".join(s)


if __name__ == "__main__":
    main()
