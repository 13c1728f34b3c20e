"""Continuous-batching server: requests that arrive while others run are
admitted and advanced together; each result equals the same request served
alone (bit for bit: members never share a reduction), and the budget is
respected."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_18042_gb300 import serve as s
    return s


def test_results_same_alone_and_in_the_mix(serve):
    reqs = serve.request_mix(10, rate=200.0, seed=7, tube=(200, 2000), quad=(32, 96), steps=(10, 40))
    stats, done = serve.run(reqs)
    assert stats["requests"] == 10 and stats["ticks"] < sum(r.steps for r in reqs)  # overlap happened
    for r in done[:6]:
        alone = serve.run_alone(r)
        assert np.array_equal(alone, r.result), r.rid
    assert stats["p99_latency_s"] >= stats["p50_latency_s"] > 0


def test_budget_limits_admission(serve):
    from paper_2511_18042_gb300 import api
    reqs = serve.request_mix(6, rate=1000.0, seed=11, tube=(300, 300), steps=(5, 10), frac_tube=1.0)
    # all requests have the same size: the state plus the solver's device scratch
    s = api.Solver.from_problem(reqs[0].prob, **serve.solver_kwargs(reqs[0].prob))
    one = s.device_bytes() + serve.state_bytes(reqs[0].prob)
    assert s.device_bytes() > 10 * serve.state_bytes(reqs[0].prob)
    del s
    stats, done = serve.run(reqs, budget_bytes=one)  # room for one request at a time
    assert stats["requests"] == 6
    # strictly sequential service: ticks equal the total number of steps
    assert stats["ticks"] == sum(r.steps for r in reqs)


def test_failed_request_is_reported_as_failed(serve):
    """Quadrant problem 249 of the seeded batch drains its four-state junction
    cell under C-GBR within 0.45 cell-crossing times (at any resolution), so
    the hybrid goes non-physical by step 20; it comes back as a failure, not a
    solve, while a request served beside it succeeds."""
    from paper_2511_18042_gb300 import inputs
    bad = inputs.batched_riemann(count=256, seed=0)[249]
    good = serve.request_mix(1, rate=1.0, seed=7, tube=(200, 400), steps=(10, 10), frac_tube=1.0)[0]
    reqs = [serve.Request(0, 0.0, bad, 25, "quad", int(bad["U"][0].size)),
            serve.Request(1, 0.0, good.prob, 10, "tube", good.cells)]
    stats, done = serve.run(reqs)
    by = {r.rid: r for r in done}
    assert by[0].status == "nonphysical" and by[1].status == "ok"
    assert stats["ok"] == 1 and stats["nonphysical"] == 1 and stats["nonphysical_ids"] == [0]
