"""The flop-counting build of the oracle (oracle/flopcount.cpp), whose counts
give the benchmark's algorithmic operations per interface, CPU only.

* Counting must not change the arithmetic: one CFL + RK3 step of the counting
  build gives the oracle's state bit for bit.
* The counts of steps with a closed form match it exactly, per cell of a 2D
  grid (nv = 4) and RK3 step:
  - primitive recovery (Sec. 2.1): 1/rho, m_k/rho, the kinetic energy and
    p = (gamma-1)(E - ke/2): 4 additions, 6 multiplications and 1 division
    a stage;
  - the TVD-RK3 combinations (Sec. 2.1): un + dt r, then 3/4 un + 1/4 (uc +
    dt r) twice: 5 additions and 7 multiplications a variable a step;
  - the residual's Jacobian scaling R = -J sum: 1 multiplication a variable
    a stage;
  - the interface flux differences, summed into the stage total: 2 additions
    a variable, a direction and a stage."""
import numpy as np
import pytest

import oracle
from paper_2511_18042_gb300 import inputs


@pytest.fixture(scope="module")
def counted():
    from oracle import count_flops as cf
    prob = inputs.triple_point(56, 24)
    U, _, _ = oracle.Oracle(prob, scheme="MEG6").advance(prob["U"], nsteps=5)
    c, Uc = cf.Counter().step(prob, U, scheme="MEG6")
    return prob, U, c, Uc


def test_counting_build_keeps_the_arithmetic(counted):
    prob, U, _, Uc = counted
    o = oracle.Oracle(prob, scheme="MEG6")
    assert np.array_equal(Uc, o.rk3_step(U, o.cfl_dt(U)))


@pytest.mark.parametrize("region,per_cell", [
    ("prim", (3 * 4, 3 * 6, 3 * 1, 0)),
    ("rk3", (4 * 5, 4 * 7, 0, 0)),
    ("residual", (0, 3 * 4, 0, 0)),
    ("flux_diff", (3 * 2 * 4 * 2, 0, 0, 0)),
])
def test_closed_form_counts(counted, region, per_cell):
    prob, _, c, _ = counted
    cells = prob["n"][0] * prob["n"][1]
    assert [v / cells for v in c[region]] == [float(x) for x in per_cell]
