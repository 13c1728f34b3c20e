"""Plain FP64 CPU oracle of the compressible-flow RHS (arXiv 2511.18042).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (``paper_2511_18042_gb300``) never imports, links or calls it.

The arithmetic lives in ``cg_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off``); this module builds it with gcc and wraps it with ctypes.
``riemann_exact`` holds the textbook exact Riemann solver used as a pin.

A function without an independent pin would be listed as "parity unpinned" in
``cg_oracle.c``'s header comment and in the design notes; every function has one.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cg_oracle.c")
_SO = os.path.join(_HERE, "_build", "libcgoracle.so")

MEG6, MIG4, LAD_E4, LAD_C6, HYBRID = 0, 1, 2, 3, 4
HYB_GLOBAL, HYB_CELL = 0, 1
BC_PERIODIC, BC_EXTRAP, BC_REFLECT, BC_INFLOW, BC_WALL = 0, 1, 2, 3, 4
SCHEMES = {"MEG6": MEG6, "MIG4": MIG4, "LAD_E4": LAD_E4, "LAD_C6": LAD_C6, "HYBRID": HYBRID}


def build(force=False):
    """Compile the oracle with gcc (plain C, no contraction of a*b+c)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("inflow", ((ctypes.c_double * 5) * 2) * 3),
        ("curvilinear", ctypes.c_int),
        ("h", ctypes.c_double * 3),
        ("period", (ctypes.c_double * 3) * 3),
        ("gamma", ctypes.c_double),
        ("minf", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("hybrid_mode", ctypes.c_int),
        ("hybrid_sensor", ctypes.c_int),
        ("hyb_rho", ctypes.c_double),
        ("hyb_p", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("c_beta", ctypes.c_double),
        ("c_kappa", ctypes.c_double),
        ("alpha_f", ctypes.c_double),
        ("sensor_thresh", ctypes.c_double),
        ("mp_eps", ctypes.c_double),
        ("mp_alpha", ctypes.c_double),
        ("read_mp_printed", ctypes.c_int),
        ("read_acoustic_mp5", ctypes.c_int),
        ("omega_window", ctypes.c_int),
        ("positivity_fallback", ctypes.c_int),
        ("filter_on", ctypes.c_int),
        ("viscous", ctypes.c_int),
        ("re", ctypes.c_double),
        ("pr", ctypes.c_double),
        ("suth", ctypes.c_double),
        ("twall", ctypes.c_double),
        ("hybrid_buffer", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        _lib.orc_create.restype = vp
        _lib.orc_create.argtypes = [ctypes.POINTER(OrcParams), P]
        _lib.orc_destroy.argtypes = [vp]
        _lib.orc_rhs.argtypes = [vp, P, P]
        _lib.orc_rk3_step.argtypes = [vp, P, ctypes.c_double]
        _lib.orc_cfl_dt.restype = ctypes.c_double
        _lib.orc_cfl_dt.argtypes = [vp, P]
        _lib.orc_hybrid_flag.restype = ctypes.c_long
        _lib.orc_hybrid_flag.argtypes = [vp, P]
        _lib.orc_omega.argtypes = [vp, P, P]
        _lib.orc_lad_coeffs.argtypes = [vp, P, P, P]
        _lib.orc_filter.argtypes = [vp, P]
        _lib.orc_metrics.argtypes = [vp, P, P]
        _lib.orc_iface_flux.argtypes = [vp, P, ctypes.c_int, P]
        _lib.orc_hllc.argtypes = [ctypes.c_int, ctypes.c_double, P, P, P, P]
        _lib.orc_euler_flux.argtypes = [ctypes.c_int, ctypes.c_double, P, P, P]
        _lib.orc_char_transform.argtypes = [ctypes.c_int, ctypes.c_double, P, P, P, ctypes.c_int, P, P]
        _lib.orc_mp5.restype = ctypes.c_double
        _lib.orc_mp5.argtypes = [ctypes.c_double] * 7
        _lib.orc_line_op.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, P, P]
        _lib.orc_tridiag.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, P, P]
        _lib.orc_set_inflow_profile.argtypes = [vp, ctypes.c_int, ctypes.c_int, P]
        _lib.orc_set_threads.restype = ctypes.c_int
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


DEFAULTS = dict(gamma=1.4, minf=1.0, scheme="MEG6", hybrid_mode=HYB_GLOBAL, hybrid_sensor=0,
                hyb_rho=-math.inf, hyb_p=-math.inf, cfl=0.2, c_beta=1.75, c_kappa=0.01,
                alpha_f=0.45, sensor_thresh=0.01, mp_eps=1e-20, mp_alpha=4.0,
                read_mp_printed=0, read_acoustic_mp5=0, omega_window=4,
                positivity_fallback=1, filter_on=1, viscous=0, re=1.0, pr=0.72, suth=0.0,
                twall=1.0, hybrid_buffer=0)


def make_params(problem, **over):
    """problem: dict with ndim, n, bc (ndim x 2), h or curvilinear info, inflow."""
    d = dict(DEFAULTS)
    d.update({k: problem[k] for k in ("gamma", "minf", "viscous", "re", "pr", "suth", "twall")
              if k in problem})
    d.update(over)
    p = OrcParams()
    nd = problem["ndim"]
    p.ndim = nd
    for k in range(3):
        p.n[k] = int(problem["n"][k]) if k < nd else 1
        p.h[k] = float(problem.get("h", [1.0, 1.0, 1.0])[k]) if k < nd else 1.0
        for s in range(2):
            p.bc[k][s] = int(problem["bc"][k][s]) if k < nd else BC_PERIODIC
            st = problem.get("inflow", {}).get((k, s))
            for v in range(5):
                p.inflow[k][s][v] = float(st[v]) if st is not None and v < len(st) else 0.0
        per = problem.get("period")
        for m in range(3):
            p.period[k][m] = float(per[k][m]) if per is not None and k < nd and m < nd else 0.0
    p.curvilinear = 1 if problem.get("xyz") is not None else 0
    p.gamma = d["gamma"]
    p.minf = d["minf"]
    s = d["scheme"]
    p.scheme = SCHEMES[s] if isinstance(s, str) else int(s)
    for k in ("hybrid_mode", "hybrid_sensor", "read_mp_printed", "read_acoustic_mp5",
              "omega_window", "positivity_fallback", "filter_on", "viscous", "hybrid_buffer"):
        setattr(p, k, int(d[k]))
    for k in ("hyb_rho", "hyb_p", "cfl", "c_beta", "c_kappa", "alpha_f", "sensor_thresh",
              "mp_eps", "mp_alpha", "re", "pr", "suth", "twall"):
        setattr(p, k, float(d[k]))
    return p


class Oracle:
    """One grid + scheme.  U arrays are (nv, nz, ny, nx)-shaped FP64 (x fastest)."""

    def __init__(self, problem, **over):
        self.problem = problem
        self.params = make_params(problem, **over)
        self.nd = problem["ndim"]
        self.nv = self.nd + 2
        self.shape = tuple(int(problem["n"][k]) for k in range(self.nd))[::-1]
        xyz = problem.get("xyz")
        self._xyz = None if xyz is None else np.ascontiguousarray(xyz, dtype=np.float64)
        L = lib()
        self._ctx = L.orc_create(ctypes.byref(self.params),
                                 None if self._xyz is None else _ptr(self._xyz))
        if not self._ctx:
            raise RuntimeError("orc_create failed")
        for (d, side), W in problem.get("inflow_profile", {}).items():
            Wp = np.ascontiguousarray(W, dtype=np.float64)
            if L.orc_set_inflow_profile(self._ctx, int(d), int(side), _ptr(Wp)) != 0:
                raise ValueError("inflow profile on a face that is not an inflow face")

    def __del__(self):
        if getattr(self, "_ctx", None):
            lib().orc_destroy(self._ctx)
            self._ctx = None

    def _arr(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (self.nv,) + self.shape, (U.shape, self.shape)
        return U

    def rhs(self, U):
        U = self._arr(U)
        R = np.empty_like(U)
        lib().orc_rhs(self._ctx, _ptr(U), _ptr(R))
        return R

    def rk3_step(self, U, dt):
        U = self._arr(U).copy()
        lib().orc_rk3_step(self._ctx, _ptr(U), float(dt))
        return U

    def cfl_dt(self, U):
        return lib().orc_cfl_dt(self._ctx, _ptr(self._arr(U)))

    def hybrid_flag(self, U):
        return int(lib().orc_hybrid_flag(self._ctx, _ptr(self._arr(U))))

    def omega(self, U):
        U = self._arr(U)
        o = np.empty(self.shape)
        lib().orc_omega(self._ctx, _ptr(U), _ptr(o))
        return o

    def lad_coeffs(self, U):
        U = self._arr(U)
        b = np.empty(self.shape)
        k = np.empty(self.shape)
        lib().orc_lad_coeffs(self._ctx, _ptr(U), _ptr(b), _ptr(k))
        return b, k

    def filter(self, U):
        U = self._arr(U).copy()
        lib().orc_filter(self._ctx, _ptr(U))
        return U

    def metrics(self):
        nd = self.nd
        node = np.empty((nd * nd + 1,) + self.shape)
        ifc = np.empty((nd * nd,) + self.shape)
        lib().orc_metrics(self._ctx, _ptr(node), _ptr(ifc))
        return node, ifc

    def iface_flux(self, U, d):
        U = self._arr(U)
        n = self.problem["n"][d]
        N = int(np.prod(self.shape))
        F = np.empty((self.nv, N // n, n + 1))
        rc = lib().orc_iface_flux(self._ctx, _ptr(U), int(d), _ptr(F))
        if rc != 0:
            raise ValueError("interface fluxes exist for the GBR schemes only")
        return F

    def advance(self, U, t_end=None, nsteps=None, dt_fixed=None):
        """March with TVD-RK3; dt from the CFL condition (clipped to t_end)."""
        t = 0.0
        k = 0
        while True:
            if nsteps is not None and k >= nsteps:
                break
            if t_end is not None and t >= t_end - 1e-14:
                break
            dt = dt_fixed if dt_fixed is not None else self.cfl_dt(U)
            if t_end is not None and t + dt > t_end:
                dt = t_end - t
            U = self.rk3_step(U, dt)
            t += dt
            k += 1
        return U, t, k


def set_threads(n=0):
    """Threads of the oracle's grid loops (0: unchanged); returns the count in
    use.  Results are the same for any count."""
    return int(lib().orc_set_threads(int(n)))


def hllc(W_L, W_R, xi, gamma=1.4):
    nd = len(xi)
    WL = np.ascontiguousarray(W_L, dtype=np.float64)
    WR = np.ascontiguousarray(W_R, dtype=np.float64)
    x = np.ascontiguousarray(xi, dtype=np.float64)
    F = np.empty(nd + 2)
    lib().orc_hllc(nd, gamma, _ptr(WL), _ptr(WR), _ptr(x), _ptr(F))
    return F


def euler_flux(W, xi, gamma=1.4):
    nd = len(xi)
    Wa = np.ascontiguousarray(W, dtype=np.float64)
    x = np.ascontiguousarray(xi, dtype=np.float64)
    F = np.empty(nd + 2)
    lib().orc_euler_flux(nd, gamma, _ptr(Wa), _ptr(x), _ptr(F))
    return F


def char_transform(W_i, W_i1, xi, w, inverse=False, gamma=1.4):
    """Characteristic variables L w (or primitive R w with inverse=True) in the
    frame of the interface between nodes with primitive states W_i, W_i1."""
    nd = len(xi)
    a, b = (np.ascontiguousarray(v, dtype=np.float64) for v in (W_i, W_i1))
    x = np.ascontiguousarray(xi, dtype=np.float64)
    wi = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty(nd + 2)
    lib().orc_char_transform(nd, gamma, _ptr(a), _ptr(b), _ptr(x), int(bool(inverse)), _ptr(wi), _ptr(out))
    return out


def mp5(um2, um1, u0, up1, up2, alpha=4.0, eps=1e-20):
    return lib().orc_mp5(um2, um1, u0, up1, up2, alpha, eps)


LINE_OPS = {"MEG6": 0, "MIG4": 1, "E4": 2, "C6": 3, "GAUSS": 4, "FILTER": 5}


def line_op(kind, f_padded, ng, periodic=False, alpha_f=0.45):
    f = np.ascontiguousarray(f_padded, dtype=np.float64)
    n = f.size - 2 * ng
    out = np.empty_like(f)
    lib().orc_line_op(LINE_OPS[kind], n, ng, int(periodic), alpha_f, _ptr(f), _ptr(out))
    return out


def tridiag(a, rhs, cyclic):
    r = np.ascontiguousarray(rhs, dtype=np.float64)
    x = np.empty_like(r)
    lib().orc_tridiag(r.size, a, int(cyclic), _ptr(r), _ptr(x))
    return x
