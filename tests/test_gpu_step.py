"""cg_step_dev (the CFL step size of U, then one RK3 step with it, the CFL
maximum reduced by stage 1's primitive kernel) equals cg_cfl_dt followed by
cg_rk3_step_dev bit for bit: the same recovery and the same rate, only one
read of the state fewer.  Every scheme and stage path (C-GBR, LAD with the
LAD-C6 filter, both hybrids, viscous curvilinear), FP64 and mixed form, over
three steps; and cg_advance, which steps through it, still matches."""
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


SCHEMES = [dict(scheme="MEG6"), dict(scheme="MIG4"), dict(scheme="LAD_E4"), dict(scheme="LAD_C6"),
           dict(scheme="HYBRID", hybrid_mode=0, hyb_rho=0.3),
           dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.3, hybrid_sensor=1, hybrid_buffer=1)]
CASES = [(kw, p) for kw in SCHEMES for p in (0, 1)]


def _bits(x):
    return x.contiguous().view(torch.int64)


def _pair(api, prob, kw, nsteps, U0=None):
    a = api.Solver.from_problem(prob, **kw)
    b = api.Solver.from_problem(prob, **kw)
    U0 = to_dev(prob["U"]) if U0 is None else U0
    Ua, Ub = U0.clone(), U0.clone()
    da = torch.zeros(2, dtype=torch.float64, device="cuda")
    db = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(nsteps):
        a.step(Ua, da)
        b.cfl_dt(Ub, out=db)
        b.rk3_step(Ub, db)
    torch.cuda.synchronize()
    sa, sb = a.sync_status(), b.sync_status()
    assert sa == sb == 0
    assert torch.equal(_bits(da[:1]), _bits(db[:1]))
    assert torch.equal(_bits(Ua), _bits(Ub))


@pytest.fixture(scope="module")
def developed(api):
    """The 112 x 48 triple point after 20 MEG6 steps (the contact and shocks
    spread over a few cells; LAD-C6 is not run from the sharp initial data)."""
    prob = inputs.triple_point(112, 48)
    U = to_dev(prob["U"])
    api.Solver.from_problem(prob, scheme="MEG6").advance(U, nsteps=20)
    torch.cuda.synchronize()
    return prob, U


@pytest.mark.parametrize("kw,precision", CASES,
                         ids=[f"{kw['scheme']}{kw.get('hybrid_mode', '')}-{'mixed' if p else 'fp64'}" for kw, p in CASES])
def test_step_equals_cfl_then_rk3_triple_point(api, developed, kw, precision):
    prob, U = developed
    _pair(api, prob, dict(kw, precision=precision), 3, U)


@pytest.mark.parametrize("kw", [SCHEMES[0], SCHEMES[3], SCHEMES[5]], ids=["MEG6", "LAD_C6", "HYBRID1"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_step_equals_cfl_then_rk3_viscous_ramp(api, kw, precision):
    ramp = inputs.compression_ramp(40, 24, 8, Lx=200.0, Ly=60.0, Lz=12.0, delta=8.0)
    _pair(api, ramp, dict(kw, precision=precision), 2)


def test_advance_matches_steps(api):
    prob = inputs.triple_point(112, 48)
    a = api.Solver.from_problem(prob, scheme="MEG6", precision=1)
    Ua, Ub = to_dev(prob["U"]), to_dev(prob["U"])
    t, k = a.advance(Ua, nsteps=4)
    d = torch.zeros(2, dtype=torch.float64, device="cuda")
    tt = 0.0
    for _ in range(4):
        a.cfl_dt(Ub, out=d)
        tt += float(d[0])
        a.rk3_step(Ub, d)
    torch.cuda.synchronize()
    assert k == 4 and abs(t - tt) <= 1e-14 * tt
    assert torch.equal(Ua, Ub)


@pytest.mark.parametrize("kw", [dict(scheme="MEG6", precision=1), dict(scheme="LAD_C6", precision=1),
                                dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.3, hybrid_sensor=1, precision=0)],
                         ids=["MEG6-mixed", "LAD_C6-mixed", "HYBRID1-fp64"])
def test_step_graph_equals_eager_steps(api, developed, kw):
    """cg_step_graph (eager first call, then a captured step replayed) gives
    the eager steps' results bit for bit, recaptures for another state tensor
    and after a tile-shape change."""
    prob, U0 = developed
    a = api.Solver.from_problem(prob, **kw)
    b = api.Solver.from_problem(prob, **kw)
    Ua, Ub, Uc = U0.clone(), U0.clone(), U0.clone()
    da = torch.zeros(2, dtype=torch.float64, device="cuda")
    db = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        for _ in range(4):
            a.step_graph(Ua, da, st)
            b.step(Ub, db, stream=st)
        for _ in range(2):  # another state: a new capture
            a.step_graph(Uc, da, st)
    st.synchronize()
    assert a.sync_status() == 0 and b.sync_status() == 0
    assert torch.equal(_bits(Ua), _bits(Ub))
    # Uc took two steps from U0 through its own capture
    Ue = U0.clone()
    with torch.cuda.stream(st):
        for _ in range(2):
            b.step(Ue, db, stream=st)
    st.synchronize()
    assert torch.equal(_bits(Uc), _bits(Ue))
    # a tile-shape change recaptures
    shape = a.tile_shape()
    a.set_tile_shape([4] * len(shape) if shape[0] != 4 else [8] * len(shape))
    Uf, Ug = U0.clone(), U0.clone()
    c = api.Solver.from_problem(prob, **kw)
    c.set_tile_shape(a.tile_shape())
    with torch.cuda.stream(st):
        for _ in range(2):
            a.step_graph(Uf, da, st)
            c.step(Ug, db, stream=st)
    st.synchronize()
    assert torch.equal(_bits(Uf), _bits(Ug))
