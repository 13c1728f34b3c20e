"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/cgflow.h.  No compute calls (CPU only)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", hdr)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"CG_API\s+[\w\s\*]+?\b(cg_\w+)\s*\(", txt)
    return names


def test_library_exports_every_declared_symbol():
    from paper_2511_18042_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_argument_errors_without_gpu():
    from paper_2511_18042_gb300 import _native as nat
    L = nat.lib()
    p = nat.CgParams()
    L.cg_params_default(ctypes.byref(p))
    assert p.gamma == 1.4 and p.cfl == 0.2 and p.c_beta == 1.75 and p.c_kappa == 0.01
    assert p.sensor_thresh == 0.01 and p.mp_eps == 1e-20 and p.omega_window == 4
    # host-side validation fails before any device work
    n = (ctypes.c_int64 * 3)(4, 1, 1)
    h = (ctypes.c_double * 3)(0.1, 1.0, 1.0)
    bc = (ctypes.c_int * 6)(1, 1, 0, 0, 0, 0)
    g = ctypes.c_void_p()
    assert L.cg_grid_create_cartesian(1, n, h, bc, ctypes.byref(g)) == -1  # n < 8 with walls
    assert b"n >= 8" in L.cg_last_error()
    n2 = (ctypes.c_int64 * 3)(16, 1, 1)
    assert L.cg_grid_create_cartesian(4, n2, h, bc, ctypes.byref(g)) == -1
    bad = (ctypes.c_int * 6)(0, 1, 0, 0, 0, 0)
    assert L.cg_grid_create_cartesian(1, n2, h, bad, ctypes.byref(g)) == -1  # half-periodic
    assert L.cg_grid_create_cartesian(1, n2, h, bc, ctypes.byref(g)) == 0
    L.cg_grid_destroy(g)


def test_solver_parameter_validation_without_gpu():
    """cg_solver_create rejects bad parameters on the host, before any device work."""
    from paper_2511_18042_gb300 import _native as nat
    L = nat.lib()
    p = nat.CgParams()
    L.cg_params_default(ctypes.byref(p))
    assert p.viscous == 0 and p.pr == 0.72 and p.twall == 1.0 and p.fma_sweep == 0 and p.precision == 0
    n = (ctypes.c_int64 * 3)(16, 1, 1)
    h = (ctypes.c_double * 3)(0.1, 1.0, 1.0)
    g = ctypes.c_void_p()
    wall = (ctypes.c_int * 6)(4, 1, 0, 0, 0, 0)  # isothermal wall, extrapolation
    assert L.cg_grid_create_cartesian(1, n, h, wall, ctypes.byref(g)) == 0
    s = ctypes.c_void_p()

    def create(**kw):
        q = nat.CgParams()
        L.cg_params_default(ctypes.byref(q))
        for k, v in kw.items():
            setattr(q, k, v)
        return L.cg_solver_create(g, ctypes.byref(q), ctypes.byref(s))

    assert create(scheme=7) == -1
    assert create(precision=3) == -1
    assert create(omega_window=5) == -1
    assert create(cfl=0.0) == -1
    assert create(viscous=1, re=0.0) == -1
    assert b"re > 0" in L.cg_last_error()
    assert create(viscous=1, re=100.0, suth=-1.0) == -1
    assert create(twall=0.0) == -1  # the grid has an isothermal wall
    assert b"twall" in L.cg_last_error()
    L.cg_grid_destroy(g)
    bad = (ctypes.c_int * 6)(5, 1, 0, 0, 0, 0)  # no boundary type 5
    assert L.cg_grid_create_cartesian(1, n, h, bad, ctypes.byref(g)) == -1


def test_empty_and_oversized_grids_rejected_without_gpu():
    from paper_2511_18042_gb300 import _native as nat
    L = nat.lib()
    h = (ctypes.c_double * 3)(0.1, 0.1, 1.0)
    per = (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0)
    g = ctypes.c_void_p()
    assert L.cg_grid_create_cartesian(2, (ctypes.c_int64 * 3)(0, 16, 1), h, per, ctypes.byref(g)) == -1  # empty
    assert L.cg_grid_create_cartesian(2, (ctypes.c_int64 * 3)(1 << 25, 16, 1), h, per, ctypes.byref(g)) == -1
    assert L.cg_grid_create_cartesian(2, (ctypes.c_int64 * 3)(16, 1, 1), h, per, ctypes.byref(g)) == 0  # one periodic line
    L.cg_grid_destroy(g)
