"""Autotuner of the sweep tile shape and of the batch stream-pool width: every
candidate tile shape gives the same right-hand side (it only regroups the same
per-interface work): bit for bit in the exact FP64 form (the default); to
rounding where the compiler fuses multiply-adds (the FMA FP64 form, FP32),
since fusion is decided per instantiation.  The tuner picks a candidate and caches it per grid shape,
and tuning a batch leaves its states unchanged."""
import itertools

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


CANDS = {0: (4, 8), 1: (4, 8, 16), 2: (4, 8, 16)}


def _cases():
    tp = inputs.triple_point(150, 70)
    xyz, per = inputs.wavy_grid_3d((20, 18, 12), amp=0.05)
    import numpy as np
    W = np.empty((5,) + xyz.shape[1:])
    W[0] = 1.0 + 0.1 * np.sin(6.28 * xyz[0])
    W[1], W[2], W[3] = 0.3, -0.2, 0.1
    W[4] = 1.0 + 0.05 * np.cos(6.28 * xyz[1])
    c3 = inputs.field_on_curvilinear(xyz, per, W)
    return [("tp_meg6_exact", tp, dict(scheme="MEG6")), ("tp_meg6_fma", tp, dict(scheme="MEG6", fma_sweep=1)),
            ("tp_mig4_exact", tp, dict(scheme="MIG4")),
            ("tp_meg6_mixed", tp, dict(scheme="MEG6", precision=1)),
            ("tp_hybrid_cell_exact", tp, dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.2, hybrid_sensor=1,
                                               )),
            ("curv3d_meg6_exact", c3, dict(scheme="MEG6")), ("curv3d_meg6_fma", c3, dict(scheme="MEG6", fma_sweep=1)),
            ("curv3d_mig4_mixed", c3, dict(scheme="MIG4", precision=1))]


def _same(a, b, kw):
    if not kw.get("fma_sweep") and not kw.get("precision"):
        return torch.equal(a, b)
    if kw.get("precision"):  # FP32: the mixed form's own metric, relative L1 per variable
        return all(float((a[v] - b[v]).abs().mean() / b[v].abs().mean()) <= 1e-5 for v in range(a.shape[0]))
    return rel_err(a, b.cpu().numpy()) <= 1e-13


@pytest.mark.parametrize("name,prob,kw", _cases(), ids=[c[0] for c in _cases()])
def test_every_tile_shape_gives_the_same_rhs(api, name, prob, kw):
    s = api.Solver.from_problem(prob, **kw)
    U = to_dev(prob["U"])
    ref = s.rhs(U)
    nd = prob["ndim"]
    shapes = list(itertools.product(*[CANDS[d] for d in range(nd)]))
    for shape in shapes:
        s.set_tile_shape(shape)
        assert _same(s.rhs(U), ref, kw), shape
    tuned = s.autotune(U, force=True)
    assert all(tuned[d] in CANDS[d] for d in range(nd))
    assert _same(s.rhs(U), ref, kw)
    # a second solver of the same shape takes the cached choice
    s2 = api.Solver.from_problem(prob, **kw)
    assert s2.autotune(U) == tuned


def test_bad_tile_shape_rejected(api):
    tp = inputs.triple_point(64, 32)
    s = api.Solver.from_problem(tp, scheme="MEG6")
    from paper_2511_18042_gb300._native import CgError
    with pytest.raises(CgError):
        s.set_tile_shape((16, 8))


def test_batch_autotune_keeps_states_and_results(api):
    probs = inputs.batched_riemann(count=12, seed=4, n_lo=24, n_hi=96)
    kw = dict(scheme="HYBRID", hybrid_mode=1, hyb_rho=0.3, hybrid_sensor=1, precision=1)
    solvers = [api.Solver.from_problem(p, **kw) for p in probs]
    Ub = [to_dev(p["U"]) for p in probs]
    stream = torch.cuda.Stream()
    batch = api.Batch(solvers, Ub)
    with torch.cuda.stream(stream):
        batch.step(stream)
        batch.step(stream)  # captured
        before = [U.clone() for U in Ub]
        width = batch.autotune(stream)
        assert width in (1, 4, 8, 16, 32)
        for a, b in zip(before, Ub):
            assert torch.equal(a, b)
        for _ in range(3):  # recapture with the tuned width, then replays
            batch.step(stream)
    stream.synchronize()
    # alone: the batch's history, two steps with the default tile shapes, then
    # three with the tuned ones (the FP32 form rounds per tile-shape instantiation)
    alone = [api.Solver.from_problem(p, **kw) for p in probs]
    Ua = [to_dev(p["U"]) for p in probs]
    for s, U in zip(alone, Ua):
        s.advance(U, nsteps=2)
    for a, m in zip(alone, solvers):
        a.set_tile_shape(m.tile_shape())
    for s, U in zip(alone, Ua):
        s.advance(U, nsteps=3)
    torch.cuda.synchronize()
    for a, b in zip(Ua, Ub):  # the mixed form's tolerance (see test_gpu_batch)
        assert torch.isfinite(b).all()
        assert float((a[0] - b[0]).abs().mean() / a[0].abs().mean()) <= 1e-5
