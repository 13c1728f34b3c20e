"""Host logic of the serving loop, on CPU: the seeded request mix (Poisson
arrivals, the 60/40 tube/quadrant split, log-uniform sizes, uniform step
counts), the per-request hybrid thresholds and the admission size estimate.
The loop itself steps on the GPU and is covered by test_gpu_serve.py."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2511_18042_gb300 import serve  # noqa: E402


def test_request_mix_is_seeded():
    a = serve.request_mix(12, rate=4.0, seed=5, tube=(50, 400), quad=(16, 48))
    b = serve.request_mix(12, rate=4.0, seed=5, tube=(50, 400), quad=(16, 48))
    for x, y in zip(a, b):
        assert (x.arrival, x.kind, x.cells, x.steps) == (y.arrival, y.kind, y.cells, y.steps)
        assert np.array_equal(x.prob["U"], y.prob["U"])
    c = serve.request_mix(12, rate=4.0, seed=6, tube=(50, 400), quad=(16, 48))
    assert [x.arrival for x in a] != [x.arrival for x in c]


def test_request_mix_defaults_within_bounds():
    reqs = serve.request_mix(24, rate=2.0, seed=1)
    for r in reqs:
        assert 50 <= r.steps <= 500
        if r.kind == "tube":
            assert r.prob["ndim"] == 1 and 200 <= r.cells <= 20000 and r.prob["U"].shape == (3, r.cells)
        else:
            n = math.isqrt(r.cells)
            assert n * n == r.cells and 128 <= n <= 1024 and r.prob["U"].shape == (4, n, n)


def test_request_mix_statistics():
    """2000 small requests: mean inter-arrival 1/rate, tube share 0.6, step
    counts uniform on [50, 500] (each within five standard errors)."""
    count, rate = 2000, 5.0
    reqs = serve.request_mix(count, rate=rate, seed=2, tube=(20, 200), quad=(8, 16))
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1.0 / rate) <= 5 * (1.0 / rate) / math.sqrt(count)
    share = np.mean([r.kind == "tube" for r in reqs])
    assert abs(share - 0.6) <= 5 * math.sqrt(0.6 * 0.4 / count)
    steps = np.array([r.steps for r in reqs])
    assert steps.min() >= 50 and steps.max() <= 500
    var = ((500 - 50 + 1) ** 2 - 1) / 12.0  # discrete uniform
    assert abs(steps.mean() - 275.0) <= 5 * math.sqrt(var / count)
    # sizes log-uniform: the mean of ln N is the midpoint of the log range
    ln_tube = np.log([r.cells for r in reqs if r.kind == "tube"])
    lo, hi = math.log(20), math.log(200)
    assert abs(ln_tube.mean() - 0.5 * (lo + hi)) <= 5 * ((hi - lo) / math.sqrt(12)) / math.sqrt(len(ln_tube)) + 0.01


def test_solver_kwargs_thresholds():
    reqs = serve.request_mix(30, rate=1.0, seed=4, tube=(50, 100), quad=(16, 24))
    seen = set()
    for r in reqs:
        kw = serve.solver_kwargs(r.prob)
        assert kw["scheme"] == "HYBRID" and kw["hybrid_mode"] == 1 and kw["hybrid_sensor"] == 1
        assert kw["precision"] == 1
        if r.kind == "tube":
            WL, WR = r.prob["WL"], r.prob["WR"]
            assert kw["hyb_rho"] == 0.5 * min(WL[0], WR[0]) and kw["hyb_p"] == 0.5 * min(WL[2], WR[2])
        else:
            st = r.prob["quad_states"]
            assert kw["hyb_rho"] == 0.5 * st[:, 0].min() and kw["hyb_p"] == 0.5 * st[:, 3].min()
        # the thresholds sit below every initial state: nothing is troubled at t = 0
        U = r.prob["U"]
        assert U[0].min() > kw["hyb_rho"]
        seen.add(r.kind)
    assert seen == {"tube", "quad"}
    assert serve.solver_kwargs(reqs[0].prob, precision=0)["precision"] == 0


def test_state_bytes_and_solver_kwargs():
    reqs = serve.request_mix(8, rate=2.0, seed=3, tube=(50, 400), quad=(16, 48))
    for r in reqs:
        nv = r.prob["ndim"] + 2
        assert serve.state_bytes(r.prob) == 8 * nv * r.cells == r.prob["U"].nbytes
        kw = serve.solver_kwargs(r.prob)
        assert kw["hybrid_mode"] == 1 and kw["hybrid_buffer"] == 1 and kw["precision"] == 1
