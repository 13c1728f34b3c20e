"""Thin Python binding of the cgflow C ABI (argument marshalling only).

Device arrays are torch CUDA tensors (FP64, contiguous, shape (nv, [nz,] [ny,] nx));
every step of the method runs in the CUDA library.  Streams are torch streams.
"""
import ctypes
import math

import torch

from . import _native as nat

SCHEMES = {"MEG6": 0, "MIG4": 1, "LAD_E4": 2, "LAD_C6": 3, "HYBRID": 4}
HYB_GLOBAL, HYB_CELL = 0, 1


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """Cartesian (h given) or curvilinear (xyz given, device tensor) structured grid."""

    def __init__(self, ndim, n, bc, h=None, xyz=None, period=None):
        L = nat.lib()
        self.ndim = ndim
        self.n = [int(n[k]) if k < ndim else 1 for k in range(3)]
        n64 = (ctypes.c_int64 * 3)(*self.n)
        bcs = (ctypes.c_int * 6)(*[int(bc[d][s]) if d < ndim else 0 for d in range(3) for s in range(2)])
        self._h = ctypes.c_void_p()
        if xyz is None:
            hh = (ctypes.c_double * 3)(*[float(h[k]) if k < ndim else 1.0 for k in range(3)])
            nat.check(L.cg_grid_create_cartesian(ndim, n64, hh, bcs, ctypes.byref(self._h)))
        else:
            xyz = xyz.to(dtype=torch.float64).contiguous()
            per = (ctypes.c_double * 9)(*[float(period[d][m]) if period is not None and d < ndim and m < ndim else 0.0
                                          for d in range(3) for m in range(3)])
            nat.check(L.cg_grid_create_curvilinear(ndim, n64, _dptr(xyz), per, bcs, ctypes.byref(self._h)))
            torch.cuda.synchronize()

    @classmethod
    def from_problem(cls, prob, device="cuda"):
        if prob.get("xyz") is not None:
            xyz = torch.as_tensor(prob["xyz"], dtype=torch.float64, device=device)
            return cls(prob["ndim"], prob["n"], prob["bc"], xyz=xyz, period=prob.get("period"))
        return cls(prob["ndim"], prob["n"], prob["bc"], h=prob["h"])

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            nat.lib().cg_grid_destroy(self._h)
            self._h = None


def make_params(scheme="MEG6", inflow=None, **kw):
    p = nat.CgParams()
    nat.lib().cg_params_default(ctypes.byref(p))
    p.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    if inflow:
        for (d, s), st in inflow.items():
            for v in range(5):
                p.inflow[d][s][v] = float(st[v]) if v < len(st) else 0.0
    return p


class Solver:
    def __init__(self, grid, scheme="MEG6", inflow=None, **kw):
        self.grid = grid
        self.params = make_params(scheme, inflow=inflow, **kw)
        self._h = ctypes.c_void_p()
        nat.check(nat.lib().cg_solver_create(grid._h, ctypes.byref(self.params), ctypes.byref(self._h)))
        self.nd = grid.ndim
        self.nv = grid.ndim + 2
        self.shape = tuple(grid.n[k] for k in range(grid.ndim))[::-1]

    @classmethod
    def from_problem(cls, prob, grid=None, **kw):
        """Solver for a problem dict (inputs module): gamma, the inflow state,
        the viscous parameters and the inflow profiles come from the problem
        unless overridden."""
        grid = grid or Grid.from_problem(prob)
        kw.setdefault("gamma", prob.get("gamma", 1.4))
        if prob.get("viscous"):
            for k in ("viscous", "re", "pr", "suth", "twall", "minf"):
                kw.setdefault(k, prob[k])
        s = cls(grid, inflow=prob.get("inflow"), **kw)
        for (d, side), W in prob.get("inflow_profile", {}).items():
            s.set_inflow_profile(d, side, W)
        return s

    def set_inflow_profile(self, d, side, W):
        """Per-node primitive profile (nv, face nodes) for inflow face (d, side)."""
        import numpy as np
        Wh = np.ascontiguousarray(W, dtype=np.float64)
        nat.check(nat.lib().cg_solver_set_inflow_profile(
            self._h, int(d), int(side), Wh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            nat.lib().cg_solver_destroy(self._h)
            self._h = None

    def _check_state(self, U):
        if tuple(U.shape) != (self.nv,) + self.shape:
            raise ValueError("state shape %s, expected %s" % (tuple(U.shape), (self.nv,) + self.shape))

    def rhs(self, U, R=None, stream=None):
        self._check_state(U)
        R = torch.empty_like(U) if R is None else R
        nat.check(nat.lib().cg_rhs(self._h, _dptr(U), _dptr(R), _stream(stream)))
        return R

    def rk3_step(self, U, dt, stream=None):
        self._check_state(U)
        if isinstance(dt, torch.Tensor):
            nat.check(nat.lib().cg_rk3_step_dev(self._h, _dptr(U), _dptr(dt), _stream(stream)))
        else:
            nat.check(nat.lib().cg_rk3_step(self._h, _dptr(U), float(dt), _stream(stream)))
        return U

    def step(self, U, dt, stream=None):
        """CFL step size of U into the device scalar dt, then one RK3 step of
        U with it (cg_step_dev: one read of U serves both)."""
        self._check_state(U)
        nat.check(nat.lib().cg_step_dev(self._h, _dptr(U), _dptr(dt), _stream(stream)))
        return U

    def step_graph(self, U, dt, stream):
        """step() replayed as a CUDA graph on a non-default stream (captured on
        the first call for these U and dt tensors, cg_step_graph)."""
        self._check_state(U)
        nat.check(nat.lib().cg_step_graph(self._h, _dptr(U), _dptr(dt), _stream(stream)))
        return U

    def cfl_dt(self, U, out=None, stream=None):
        self._check_state(U)
        if out is not None:
            nat.check(nat.lib().cg_cfl_dt(self._h, _dptr(U), _dptr(out), 1, _stream(stream)))
            return out
        v = ctypes.c_double()
        nat.check(nat.lib().cg_cfl_dt(self._h, _dptr(U), ctypes.byref(v), 0, _stream(stream)))
        return v.value

    def autotune(self, U, force=False, stream=None):
        """Choose the sweep tile shape by timing the RHS of U (cached per shape);
        returns the lines per tile per direction."""
        self._check_state(U)
        nat.check(nat.lib().cg_autotune(self._h, _dptr(U), int(bool(force)), _stream(stream)))
        return self.tile_shape()

    def tile_shape(self):
        lw = (ctypes.c_int * 3)()
        nat.check(nat.lib().cg_tile_shape(self._h, lw))
        return tuple(lw[: self.nd])

    def set_tile_shape(self, shape):
        lw = (ctypes.c_int * 3)(*(list(shape) + [0] * (3 - len(shape))))
        nat.check(nat.lib().cg_set_tile_shape(self._h, lw))

    def advance(self, U, nsteps=0, t_end=0.0, stream=None):
        self._check_state(U)
        t = ctypes.c_double()
        k = ctypes.c_int64()
        nat.check(nat.lib().cg_advance(self._h, _dptr(U), int(nsteps), float(t_end), ctypes.byref(t),
                                       ctypes.byref(k), _stream(stream)))
        return t.value, k.value

    def advance_host(self, U_host, nsteps=0, t_end=0.0, stream=None):
        """U_host: pinned (or pageable) CPU float64 tensor, updated in place."""
        if U_host.is_cuda or U_host.dtype != torch.float64 or not U_host.is_contiguous():
            raise ValueError("expected a contiguous float64 CPU tensor")
        t = ctypes.c_double()
        nat.check(nat.lib().cg_advance_host(self._h, ctypes.c_void_p(U_host.data_ptr()), int(nsteps), float(t_end),
                                            ctypes.byref(t), _stream(stream)))
        return t.value

    def omega(self, U, stream=None):
        out = torch.empty(self.shape, dtype=torch.float64, device=U.device)
        nat.check(nat.lib().cg_omega(self._h, _dptr(U), _dptr(out), _stream(stream)))
        return out

    def lad_coeffs(self, U, stream=None):
        b = torch.empty(self.shape, dtype=torch.float64, device=U.device)
        k = torch.empty_like(b)
        nat.check(nat.lib().cg_lad_coeffs(self._h, _dptr(U), _dptr(b), _dptr(k), _stream(stream)))
        return b, k

    def filter(self, U, stream=None):
        nat.check(nat.lib().cg_filter(self._h, _dptr(U), _stream(stream)))
        return U

    def iface_flux(self, U, d, stream=None):
        n = self.grid.n[d]
        N = 1
        for s in self.shape:
            N *= s
        F = torch.empty((self.nv, N // n, n + 1), dtype=torch.float64, device=U.device)
        nat.check(nat.lib().cg_iface_flux(self._h, _dptr(U), int(d), _dptr(F), _stream(stream)))
        return F

    def metrics(self, stream=None):
        dev = torch.device("cuda")
        node = torch.empty((self.nd * self.nd + 1,) + self.shape, dtype=torch.float64, device=dev)
        ifc = torch.empty((self.nd * self.nd,) + self.shape, dtype=torch.float64, device=dev)
        nat.check(nat.lib().cg_metrics(self._h, _dptr(node), _dptr(ifc), _stream(stream)))
        return node, ifc

    def hybrid_state(self, stream=None):
        f = ctypes.c_int()
        n = ctypes.c_int64()
        nat.check(nat.lib().cg_hybrid_state(self._h, ctypes.byref(f), ctypes.byref(n), _stream(stream)))
        return f.value, n.value

    def sync_status(self, stream=None):
        return nat.lib().cg_sync_status(self._h, _stream(stream))

    def launch_count(self):
        return int(nat.lib().cg_launch_count(self._h))

    def device_bytes(self):
        """Device memory the solver holds (scratch; the caller's state excluded)."""
        return int(nat.lib().cg_solver_device_bytes(self._h))

    def timing_enable(self, on=True):
        nat.check(nat.lib().cg_timing_enable(self._h, 1 if on else 0))

    def timing_query(self, kernel_class=0):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        nat.check(nat.lib().cg_timing_query(self._h, int(kernel_class), ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


def multi_step(solvers, states, stream=None):
    """One RK3 step (own CFL dt) of every solver on its state, concurrently."""
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s._h.value for s in solvers])
    ps = (ctypes.c_void_p * n)(*[U.data_ptr() for U in states])
    for s, U in zip(solvers, states):
        s._check_state(U)
    nat.check(nat.lib().cg_multi_step(hs, ps, n, _stream(stream)))


class Batch:
    """A fixed set of (solver, state) pairs stepped together; from the second
    step on, one CUDA graph replay per step (needs a non-default stream)."""

    def __init__(self, solvers, states):
        self.solvers = list(solvers)
        self.states = list(states)
        for s, U in zip(self.solvers, self.states):
            s._check_state(U)
        n = len(self.solvers)
        hs = (ctypes.c_void_p * n)(*[s._h.value for s in self.solvers])
        ps = (ctypes.c_void_p * n)(*[U.data_ptr() for U in self.states])
        self._h = ctypes.c_void_p()
        nat.check(nat.lib().cg_batch_create(n, hs, ps, ctypes.byref(self._h)))

    def step(self, stream):
        nat.check(nat.lib().cg_batch_step(self._h, _stream(stream)))

    def autotune(self, stream=None):
        """Tile shapes of the members and the stream-pool width (states unchanged);
        returns the chosen width."""
        w = ctypes.c_int()
        nat.check(nat.lib().cg_batch_autotune(self._h, _stream(stream), ctypes.byref(w)))
        return w.value

    def path(self):
        """("persistent", 3) on the persistent stages, ("table", launches per
        step) on the work-table path, ("streams", None) on the stream pool."""
        p, n = ctypes.c_int(), ctypes.c_int()
        nat.check(nat.lib().cg_batch_path(self._h, ctypes.byref(p), ctypes.byref(n)))
        return {2: ("persistent", n.value), 1: ("table", n.value)}.get(p.value, ("streams", None))

    def set_path(self, path, groups=1):
        """path: "streams", "table" (in `groups` member groups) or "persistent"."""
        code = {"streams": 0, "table": 1, "persistent": 2}[path]
        nat.check(nat.lib().cg_batch_set_path(self._h, code, int(groups)))

    def sync(self, stream=None):
        """Synchronise; raises if a persistent stage's barrier wait ran out."""
        nat.check(nat.lib().cg_batch_sync(self._h, _stream(stream)))

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            nat.lib().cg_batch_destroy(self._h)
            self._h = None
