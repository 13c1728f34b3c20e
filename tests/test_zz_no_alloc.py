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


@pytest.mark.parametrize("case", ["triple_point", "sod"])
def test_noalloc_rhs_matches_solver_rhs_twice(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18042_gb300 import _native as nat
    from paper_2511_18042_gb300 import api
    L = nat.lib()
    L.cg_rhs_meg6_noalloc.restype = ctypes.c_int
    L.cg_rhs_meg6_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(nat.CgParams), ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
    prob = inputs.triple_point(224, 96) if case == "triple_point" else inputs.shock_tube("sod", 400)
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


def test_noalloc_rejects_large_grids():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18042_gb300 import _native as nat
    from paper_2511_18042_gb300 import api
    L = nat.lib()
    L.cg_rhs_meg6_noalloc.restype = ctypes.c_int
    L.cg_rhs_meg6_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(nat.CgParams), ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
    prob = inputs.triple_point(512, 256)  # 131072 cells
    params = api.make_params("MEG6")
    U = torch.as_tensor(prob["U"], device="cuda")
    R = torch.empty_like(U)
    rc = _call(L, prob, params, U, R)
    assert rc == -1
    assert b"too large" in L.cg_last_error()
