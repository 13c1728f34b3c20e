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
    reqs = serve.request_mix(6, rate=1000.0, seed=11, tube=(300, 300), steps=(5, 10), frac_tube=1.0)
    one = serve.bytes_estimate(reqs[0].prob)  # all requests have the same size
    stats, done = serve.run(reqs, budget_bytes=one)  # room for one request at a time
    assert stats["requests"] == 6
    # strictly sequential service: ticks equal the total number of steps
    assert stats["ticks"] == sum(r.steps for r in reqs)
