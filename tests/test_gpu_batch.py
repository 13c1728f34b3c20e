"""Batched advance of uneven grids (cg_multi_step / cg_batch with CUDA-graph
replay): every member's result equals the same member advanced alone (bit for
bit in FP64; in the mixed form within its tolerance, a density L1 of 1e-5: the
batched FP32 kernels are other instantiations of the same code, and the
compiler may fuse their multiply-adds differently), and a member matches the
oracle."""
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


def same_member(alone, batched, kw):
    """FP64: bit for bit; mixed form: density L1 within 1e-5 of the member alone."""
    if kw.get("precision", 0) == 0:
        assert torch.equal(alone, batched)
        return
    assert torch.isfinite(batched).all()
    ra, rb = alone[0], batched[0]
    assert float((ra - rb).abs().mean() / ra.abs().mean()) <= 1e-5


KW = [dict(scheme="MEG6"), dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.3, hybrid_sensor=1),
      dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.3, hybrid_sensor=1, precision=1),
      dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.3, hybrid_sensor=1, hybrid_buffer=1)]


@pytest.mark.parametrize("kw", KW)
def test_batch_equals_members_alone(api, kw):
    probs = inputs.batched_riemann(count=10, seed=3, n_lo=24, n_hi=90)
    solvers = [api.Solver.from_problem(p, **kw) for p in probs]
    alone = [api.Solver.from_problem(p, **kw) for p in probs]
    Ub = [to_dev(p["U"]) for p in probs]
    Ua = [to_dev(p["U"]) for p in probs]
    stream = torch.cuda.Stream()
    batch = api.Batch(solvers, Ub)
    with torch.cuda.stream(stream):
        for _ in range(5):  # eager, capture + replay, replays
            batch.step(stream)
    stream.synchronize()
    for s, U in zip(alone, Ua):
        s.advance(U, nsteps=5)
    torch.cuda.synchronize()
    for a, b in zip(Ua, Ub):
        same_member(a, b, kw)
    # 2D Cartesian per-interface hybrids step through the work table
    want = "table" if kw.get("hybrid_mode") == 1 else "streams"
    assert batch.path()[0] == want


def test_work_table_after_autotune(api):
    """The autotuner may move a qualifying batch to one common tile shape and
    a few concurrent member groups; members then match members alone with that
    shape, and the table's launch count does not grow with the member count."""
    kw = dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.3, hybrid_sensor=1, precision=1)
    probs = inputs.batched_riemann(count=24, seed=7, n_lo=20, n_hi=130)
    solvers = [api.Solver.from_problem(p, **kw) for p in probs]
    Ub = [to_dev(p["U"]) for p in probs]
    stream = torch.cuda.Stream()
    batch = api.Batch(solvers, Ub)
    batch.autotune(stream)
    with torch.cuda.stream(stream):
        for _ in range(4):
            batch.step(stream)
    stream.synchronize()
    path, launches = batch.path()
    alone = []
    for p, s in zip(probs, solvers):
        a = api.Solver.from_problem(p, **kw)
        a.set_tile_shape(s.tile_shape())
        U = to_dev(p["U"])
        a.advance(U, nsteps=4)
        alone.append(U)
    torch.cuda.synchronize()
    for a, b in zip(alone, Ub):
        same_member(a, b, kw)
    if path == "table":
        assert launches in (41, 82, 164, 328)  # 41 per member group
    if path == "persistent":
        assert launches == 3  # one cooperative launch per RK stage


def test_multi_step_member_matches_oracle(orc, api):
    probs = inputs.batched_riemann(count=6, seed=5, n_lo=24, n_hi=70)
    solvers = [api.Solver.from_problem(p, scheme="MEG6") for p in probs]
    Us = [to_dev(p["U"]) for p in probs]
    for _ in range(10):
        api.multi_step(solvers, Us)
    torch.cuda.synchronize()
    for p, U in zip(probs[:2], Us[:2]):
        o = orc.Oracle(p, scheme="MEG6")
        Uo, _, _ = o.advance(p["U"], nsteps=10)
        assert rel_err(U, Uo) <= 1e-11


def test_full_batch_sampled_members(api):
    """The batched workload at full size, as the benchmark runs it: 256 quadrant
    problems (64^2..512^2, seed 0), per-interface hybrid in the mixed form,
    autotuned batch (work table or stream pool), graph replays; eight sampled
    members match the same members advanced alone with their tuned tile shapes."""
    from bench import _hybrid_kw
    probs = inputs.batched_riemann(count=256, seed=0)
    solvers = [api.Solver.from_problem(p, **_hybrid_kw(p, 1)) for p in probs]
    Ub = [to_dev(p["U"]) for p in probs]
    stream = torch.cuda.Stream()
    batch = api.Batch(solvers, Ub)
    with torch.cuda.stream(stream):
        batch.autotune(stream)
        for _ in range(4):  # eager, capture, replays
            batch.step(stream)
    stream.synchronize()
    rng = np.random.default_rng(1)
    for m in sorted(rng.choice(len(probs), size=8, replace=False)):
        a = api.Solver.from_problem(probs[m], **_hybrid_kw(probs[m], 1))
        a.set_tile_shape(solvers[m].tile_shape())
        U = to_dev(probs[m]["U"])
        a.advance(U, nsteps=4)
        torch.cuda.synchronize()
        same_member(U, Ub[m], dict(precision=1))


@pytest.mark.parametrize("kw", [KW[1], KW[3], KW[2]], ids=["fp64", "fp64_buffer", "mixed"])
def test_persistent_stages_equal_members_alone(api, kw):
    """One cooperative launch per RK stage (the work table's phases with grid
    barriers between them): every member equals the member stepped alone,
    bitwise in FP64, within the mixed tolerance in the mixed form."""
    probs = inputs.batched_riemann(count=10, seed=3, n_lo=24, n_hi=90)
    solvers = [api.Solver.from_problem(p, **kw) for p in probs]
    alone = [api.Solver.from_problem(p, **kw) for p in probs]
    Ub = [to_dev(p["U"]) for p in probs]
    Ua = [to_dev(p["U"]) for p in probs]
    stream = torch.cuda.Stream()
    batch = api.Batch(solvers, Ub)
    batch.set_path("persistent")
    with torch.cuda.stream(stream):
        for _ in range(5):  # eager, capture + replay, replays
            batch.step(stream)
    batch.sync(stream)
    assert batch.path() == ("persistent", 3)
    for s, U in zip(alone, Ua):
        s.advance(U, nsteps=5)
    torch.cuda.synchronize()
    for a, b in zip(Ua, Ub):
        same_member(a, b, kw)
    # and back to the table's launches: the same members again
    batch.set_path("table")
    with torch.cuda.stream(stream):
        for _ in range(3):
            batch.step(stream)
    batch.sync(stream)
    assert batch.path()[0] == "table"


def test_persistent_barrier_wait_is_bounded(api):
    """A barrier that waits for an arrival that never comes gives up after
    about a second, the launch ends, and cg_batch_sync reports CG_ERR_TIMEOUT;
    with the normal count restored the batch steps again."""
    import ctypes
    from paper_2511_18042_gb300 import _native as nat
    kw = KW[1]
    probs = inputs.batched_riemann(count=3, seed=3, n_lo=24, n_hi=40)
    solvers = [api.Solver.from_problem(p, **kw) for p in probs]
    Ub = [to_dev(p["U"]) for p in probs]
    stream = torch.cuda.Stream()
    batch = api.Batch(solvers, Ub)
    batch.set_path("persistent")
    assert nat.lib().cg_batch_debug_barrier(batch._h, 1) == 0
    with torch.cuda.stream(stream):
        batch.step(stream)  # eager: three stages, each ends at its first barrier
    rc = nat.lib().cg_batch_sync(batch._h, ctypes.c_void_p(stream.cuda_stream))
    assert rc == -6, nat.lib().cg_last_error()
    assert nat.lib().cg_batch_debug_barrier(batch._h, 0) == 0
    for U, p in zip(Ub, probs):
        U.copy_(to_dev(p["U"]))
    with torch.cuda.stream(stream):
        for _ in range(3):
            batch.step(stream)
    batch.sync(stream)
    assert all(torch.isfinite(U).all() for U in Ub)
