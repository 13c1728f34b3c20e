"""The no-allocation MEG6 RHS (cg_rhs_meg6_noalloc) gives the same result as
the solver-based cg_rhs, on two calls in a row.

It serves callers that cannot allocate device memory (code inside a CUDA graph
capture, plug-ins whose host owns all device memory, real-time loops); its
working arrays live in a fixed device array of the library.  The test calls it
through the C ABI with ctypes, in its own file so that pytest runs it last."""
import ctypes

import numpy as np
import pytest

from paper_2511_18042_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _call(L, prob, params, U, R):
    nd = prob["ndim"]
    n = (ctypes.c_int64 * 3)(*[int(prob["n"][k]) if k < nd else 1 for k in range(3)])
    h = (ctypes.c_double * 3)(*[float(prob["h"][k]) if k < nd else 1.0 for k in range(3)])
    bc = (ctypes.c_int * 6)(*[int(prob["bc"][d][s]) if d < nd else 0 for d in range(3) for s in range(2)])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.cg_rhs_meg6_noalloc(nd, n, h, bc, ctypes.byref(params), ctypes.c_void_p(U.data_ptr()),
                                 ctypes.c_void_p(R.data_ptr()), stream)


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18042_gb300 import _native as nat
    L = nat.lib()
    L.cg_rhs_meg6_noalloc.restype = ctypes.c_int
    L.cg_rhs_meg6_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(nat.CgParams), ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
    return L


def _box3d(nx=32, ny=24, nz=16):
    """3D Cartesian box: reflective walls in x, periodic y, extrapolation in z,
    a smooth state with a pressure step (the sensor and MP5 both act)."""
    h = [1.0 / nx, 0.75 / ny, 0.5 / nz]
    z, y, x = np.meshgrid(*[(np.arange(n) + 0.5) * hh for n, hh in ((nz, h[2]), (ny, h[1]), (nx, h[0]))],
                          indexing="ij")
    W = np.stack([1.0 + 0.2 * np.sin(2 * np.pi * y / 0.75) * np.cos(3 * x), 0.3 * np.sin(np.pi * x),
                  0.2 * np.cos(2 * np.pi * y / 0.75), 0.1 * np.sin(4 * z), np.where(x < 0.5, 1.0, 0.4)])
    return inputs._problem("box3d", 3, [nx, ny, nz], h, [[2, 2], [0, 0], [1, 1]], W, 1.4)


@pytest.mark.parametrize("case", ["triple_point", "sod", "box3d"])
def test_noalloc_rhs_matches_solver_rhs_twice(case):
    L = _lib()
    from paper_2511_18042_gb300 import api
    prob = {"triple_point": lambda: inputs.triple_point(224, 96), "sod": lambda: inputs.shock_tube("sod", 400),
            "box3d": _box3d}[case]()
    solver = api.Solver.from_problem(prob, scheme="MEG6")
    params = api.make_params("MEG6", inflow=prob.get("inflow"), gamma=prob["gamma"])
    U0 = torch.as_tensor(prob["U"], device="cuda")
    U1 = U0.clone()
    solver.advance(U1, nsteps=10)  # a second, developed state
    for U in (U0, U1):  # two calls in a row, the scratch array reused
        R = torch.full_like(U, float("nan"))
        assert _call(L, prob, params, U, R) == 0, L.cg_last_error()
        ref = solver.rhs(U)
        torch.cuda.synchronize()
        scale = ref.abs().amax(dim=tuple(range(1, ref.dim())), keepdim=True).clamp_min(1e-300)
        assert float(((R - ref).abs() / scale).max()) <= 1e-13


@pytest.mark.parametrize("kw,bc,code", [
    (dict(scheme="MEG6", viscous=1, re=100.0), None, -5),   # inviscid only
    (dict(scheme="MEG6", precision=1), None, -5),           # FP64 only
    (dict(scheme="LAD_E4"), None, -5),                      # MEG6 only
    (dict(scheme="MEG6", minf=0.0), None, -1),              # checked as by cg_solver_create
    (dict(scheme="MEG6", twall=0.0), [[4, 2], [2, 2]], -1), # isothermal wall needs twall > 0
    (dict(scheme="MEG6", omega_window=5), None, -1),
])
def test_noalloc_rejects_unsupported_parameters(kw, bc, code):
    """Refused before any launch, with the same codes as cg_solver_create."""
    L = _lib()
    from paper_2511_18042_gb300 import api
    prob = inputs.triple_point(64, 32)
    if bc is not None:
        prob["bc"] = bc
    params = api.make_params(**kw)
    U = torch.as_tensor(prob["U"], device="cuda")
    R = torch.empty_like(U)
    assert _call(L, prob, params, U, R) == code, L.cg_last_error()


def test_noalloc_rejects_large_grids():
    L = _lib()
    from paper_2511_18042_gb300 import api
    prob = inputs.triple_point(512, 256)  # 131072 cells
    params = api.make_params("MEG6")
    U = torch.as_tensor(prob["U"], device="cuda")
    R = torch.empty_like(U)
    rc = _call(L, prob, params, U, R)
    assert rc == -1
    assert b"too large" in L.cg_last_error()
