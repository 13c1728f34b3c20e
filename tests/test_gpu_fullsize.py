"""The bench workloads at their full sizes, in the launch configuration the
benchmark times (autotuned tile shapes, default FP64 form):

* triple point 1792 x 768: one RK3 step of each of the six schemes from a
  state the oracle developed (5 MEG6 steps from the initial condition),
  compared element by element with the oracle's step, and 100 steps of MEG6
  and the per-interface hybrid from the initial condition;
* compression-ramp grid 768 x 192 x 128: a uniform stream through the full
  body-fitted grid (inflow and outflow at the free-stream state, the wall
  replaced by extrapolation) stays uniform to round-off for every scheme,
  inviscid and viscous (the discrete metric identities hold at full size)."""
import numpy as np
import pytest

from paper_2511_18042_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from tests.gpu_util import rel_err, to_dev  # noqa: E402


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18042_gb300 import api as a
    return a


SIX = [("MEG6", dict(scheme="MEG6")), ("MIG4", dict(scheme="MIG4")), ("LAD_E4", dict(scheme="LAD_E4")),
       ("LAD_C6", dict(scheme="LAD_C6")), ("HYBRID_GLOBAL", dict(scheme="HYBRID", hybrid_mode=0, hyb_rho=0.0625)),
       ("HYBRID_CELL", dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.0625, hybrid_sensor=1))]


@pytest.fixture(scope="module")
def developed(orc):
    prob = inputs.triple_point()
    o = orc.Oracle(prob, scheme="MEG6")
    U, _, _ = o.advance(prob["U"], nsteps=5)
    return prob, U


@pytest.mark.parametrize("name,kw", SIX, ids=[n for n, _ in SIX])
def test_triple_point_full_size_every_scheme(orc, api, developed, name, kw):
    prob, U = developed
    o = orc.Oracle(prob, **kw)
    s = api.Solver.from_problem(prob, **kw)
    Ud = to_dev(U)
    s.autotune(Ud)
    dt_o = o.cfl_dt(U)
    dt = torch.zeros(2, dtype=torch.float64, device="cuda")
    s.cfl_dt(Ud, out=dt)
    assert abs(float(dt[0]) - dt_o) <= 1e-14 * dt_o
    s.rk3_step(Ud, dt_o)
    Uo = o.rk3_step(U, dt_o)
    assert rel_err(Ud, Uo) <= 1e-12, name


@pytest.mark.parametrize("name", ["MEG6", "HYBRID_CELL"])
def test_triple_point_full_size_100_steps(orc, api, name):
    """The spec bar at the benchmark's size: 100 RK3 steps (CFL time
    steps on each side) of the 1792 x 768 triple point from its initial
    condition, max relative error <= 1e-11 per variable against the oracle
    (run on all host cores; its results do not depend on the thread count)."""
    kw = dict(SIX)[name]
    prob = inputs.triple_point()
    orc.set_threads(0)
    Uo, to, ko = orc.Oracle(prob, **kw).advance(prob["U"], nsteps=100)
    s = api.Solver.from_problem(prob, **kw)
    Ud = to_dev(prob["U"])
    s.autotune(Ud)
    tg, kg = s.advance(Ud, nsteps=100)
    assert kg == ko == 100 and abs(tg - to) <= 1e-13 * to
    assert rel_err(Ud, Uo) <= 1e-11, name


@pytest.mark.parametrize("viscous", [False, True])
def test_full_ramp_grid_preserves_a_uniform_stream(api, viscous):
    ramp = inputs.compression_ramp()
    W0 = (1.0, 1.0, 0.2, -0.1, 1.0 / (1.4 * 2.9 ** 2))
    n = ramp["n"]
    W = np.empty((5, n[2], n[1], n[0]))
    for v in range(5):
        W[v] = W0[v]
    prob = inputs._problem("ramp_uniform", 3, n, [1.0] * 3,
                           [[inputs.INFLOW, inputs.EXTRAP], [inputs.EXTRAP, inputs.EXTRAP],
                            [inputs.PERIODIC, inputs.PERIODIC]], W, 1.4,
                           xyz=ramp["xyz"], period=ramp["period"])
    prob["inflow"] = {(0, 0): W0}
    if viscous:
        prob = inputs._viscous(prob, 2400.0, 2.9, ramp["suth"], ramp["t_wall"])
    U = to_dev(prob["U"])
    grid = api.Grid.from_problem(prob)
    scale = float(U.abs().max())
    # cell volumes from the node spacings (J ~ 1/volume), for a per-volume residual
    x, y = ramp["xyz"][0], ramp["xyz"][1]
    dx = np.diff(x, axis=2, append=2 * x[:, :, -1:] - x[:, :, -2:-1])
    dy = np.diff(y, axis=1, append=2 * y[:, -1:, :] - y[:, -2:-1, :])
    vol = torch.as_tensor(np.abs(dx * dy) * (ramp["period"][2][2] / n[2]), device="cuda")
    for kw in (dict(scheme="MEG6"), dict(scheme="MIG4"), dict(scheme="LAD_E4"),
               dict(scheme="HYBRID", hybrid_mode=1, hybrid_sensor=1, hyb_rho=0.5)):
        s = api.Solver.from_problem(prob, grid=grid, **kw)
        R = s.rhs(U)
        # residual times the cell volume (the flux balance of the cell) against the state scale
        worst = float((R * vol.unsqueeze(0)).abs().max()) / scale
        assert worst <= 1e-10, (kw, worst)
        del s, R
        torch.cuda.empty_cache()
