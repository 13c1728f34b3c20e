"""Mixed precision form (FP32 reconstruction and fluxes, FP64 primitive
recovery and RK accumulation) against the FP64 oracle.  Tolerance: density L1
(mean absolute difference) <= 1e-5 on shocked 2D cases after 100 RK3 steps,
and the same on the Sod tube at t = 0.2."""
import math

import numpy as np
import pytest

from paper_2511_18042_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from tests.gpu_util import to_dev  # noqa: E402


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18042_gb300 import api as a
    return a


def _l1_rho(Ug, Uo):
    return float(np.abs(Ug[0].cpu().numpy() - Uo[0]).mean())


@pytest.mark.parametrize("kw", [dict(scheme="MEG6"), dict(scheme="MIG4"), dict(scheme="LAD_E4"),
                                dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.0625, hybrid_sensor=1),
                                dict(scheme="HYBRID", hybrid_mode=0, hyb_rho=0.12)])
def test_mixed_triple_point_100_steps(orc, api, kw):
    prob = inputs.triple_point(224, 96)
    o = orc.Oracle(prob, **kw)
    Uo, _, _ = o.advance(prob["U"], nsteps=100)
    s = api.Solver.from_problem(prob, precision=1, **kw)
    Ug = to_dev(prob["U"])
    s.advance(Ug, nsteps=100)
    err = _l1_rho(Ug, Uo)
    assert err <= 1e-5, err
    assert torch.isfinite(Ug).all()


def test_mixed_sod(orc, api):
    prob = inputs.shock_tube("sod", 400)
    o = orc.Oracle(prob, scheme="MEG6", cfl=0.5)
    Uo, _, _ = o.advance(prob["U"], t_end=0.2)
    s = api.Solver.from_problem(prob, scheme="MEG6", precision=1, cfl=0.5)
    Ug = to_dev(prob["U"])
    s.advance(Ug, t_end=0.2)
    assert _l1_rho(Ug, Uo) <= 1e-5


def test_mixed_rhs_close_to_fp64(orc, api):
    prob = inputs.triple_point(224, 96)
    pre = orc.Oracle(prob, scheme="MEG6")
    U, _, _ = pre.advance(prob["U"], nsteps=30)
    s = api.Solver.from_problem(prob, scheme="MEG6", precision=1)
    R = s.rhs(to_dev(U)).cpu().numpy()
    Ro = pre.rhs(U)
    for v in range(4):
        assert np.abs(R[v] - Ro[v]).max() <= 1e-4 * np.abs(Ro[v]).max()


def test_mixed_sensor_close_to_fp64(orc, api):
    """The mixed form keeps the discontinuity sensor of Eq. (8) in FP32. Read back through
    the diagnostics call it stays within FP32 rounding of the oracle's sensor
    (values up to ~0.4 here) on a shocked state."""
    prob = inputs.riemann_c3(48)
    o = orc.Oracle(prob, scheme="MEG6")
    U, _, _ = o.advance(prob["U"], nsteps=10)
    om_o = o.omega(U)
    assert om_o.max() > 0.2
    s = api.Solver.from_problem(prob, scheme="MEG6", precision=1)
    om = s.omega(to_dev(U)).cpu().numpy()
    d = np.abs(om - om_o)
    assert d.max() <= 1e-2 and d.mean() <= 1e-4, (d.max(), d.mean())


@pytest.mark.parametrize("scheme", ["LAD_C6", "LAD_E4"])
def test_mixed_lad_sod(orc, api, scheme):
    """LAD in the mixed form on the Sod tube (N = 400, long quiet region ahead of
    the shock). LAD-C6: FP32 compact derivatives of the fields and the fluxes,
    FP64 implicit filter of the state; the compact derivatives' tails there
    reach 1e-22..1e-32, where an FP32 sum of squares in |grad rho| flushes."""
    prob = inputs.shock_tube("sod", 400)
    o = orc.Oracle(prob, scheme=scheme, cfl=0.1)
    Uo, _, _ = o.advance(prob["U"], t_end=0.2)
    s = api.Solver.from_problem(prob, scheme=scheme, precision=1, cfl=0.1)
    Ug = to_dev(prob["U"])
    s.advance(Ug, t_end=0.2)
    assert torch.isfinite(Ug).all()
    assert _l1_rho(Ug, Uo) <= 1e-5


def test_mixed_lad_c6_periodic_2d(orc, api):
    prob = inputs.kelvin_helmholtz(64)
    o = orc.Oracle(prob, scheme="LAD_C6", cfl=0.1)
    Uo, _, _ = o.advance(prob["U"], nsteps=50)
    s = api.Solver.from_problem(prob, scheme="LAD_C6", precision=1, cfl=0.1)
    Ug = to_dev(prob["U"])
    s.advance(Ug, nsteps=50)
    assert _l1_rho(Ug, Uo) <= 1e-5
    assert torch.isfinite(Ug).all()


@pytest.mark.parametrize("kw", [dict(scheme="MEG6"), dict(scheme="MIG4"), dict(scheme="LAD_E4"),
                                dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.8, hybrid_sensor=1)])
def test_mixed_curvilinear_2d(orc, api, kw):
    """The mixed form on a periodic 2D curvilinear grid (metrics in FP64, read
    by the FP32 kernels): density L1 against the oracle after 20 steps <= 1e-5."""
    xyz, per = inputs.wavy_grid_2d(40, 36, amp=0.08)
    x, y = xyz
    W = np.stack([1.0 + 0.3 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y), 0.5 + 0 * x,
                  0.2 + 0.1 * np.cos(2 * math.pi * y), 1.0 + 0.2 * np.sin(2 * math.pi * (x + y))])
    prob = inputs.field_on_curvilinear(xyz, per, W)
    o = orc.Oracle(prob, **kw)
    Uo, _, _ = o.advance(prob["U"], nsteps=20)
    s = api.Solver.from_problem(prob, precision=1, **kw)
    Ug = to_dev(prob["U"])
    s.advance(Ug, nsteps=20)
    assert torch.isfinite(Ug).all()
    rho = Ug[0].cpu().numpy()
    assert np.abs(rho - Uo[0]).mean() / np.abs(Uo[0]).mean() <= 1e-5, kw
