"""Pins of LAD-C6 on curvilinear grids (Sec. 2.1 metrics, Sec. 2.2 LAD-C6,
Algorithm 1 filter), CPU only.

The metrics of LAD-C6 are built with its own compact sixth-order operator
(the operator of its flux divergence), so the discrete metric identities hold
for it: a uniform stream stays uniform to round-off on wavy and body-fitted
grids.  The implicit filter acts on the transformed conserved vector Q/J on a
curvilinear grid, so the discrete conservation of sum(Q/J) survives it.  And
the metric operator really is the compact one: on a smooth periodic wavy grid
the metrics converge to the analytic ones at sixth order (E4 metrics at
fourth)."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_18042_gb300 import inputs


def _analytic_wavy_2d(nx, ny, amp, Lx=1.0, Ly=1.0):
    """Exact xi_hat = (y_eta, -x_eta), eta_hat = (-y_xi, x_xi) of
    inputs.wavy_grid_2d in index space (xi = i, eta = j)."""
    I, J = np.meshgrid(np.arange(nx), np.arange(ny))
    a, b = 2 * math.pi * I / nx, 2 * math.pi * J / ny
    x_xi = Lx * (1.0 / nx + amp * (2 * math.pi / nx) * np.cos(a) * np.sin(b))
    x_eta = Lx * amp * (2 * math.pi / ny) * np.sin(a) * np.cos(b)
    y_xi = Ly * amp * (2 * math.pi / nx) * np.cos(a) * np.sin(b)
    y_eta = Ly * (1.0 / ny + amp * (2 * math.pi / ny) * np.sin(a) * np.cos(b))
    return np.stack([y_eta, -x_eta, -y_xi, x_xi])


@pytest.mark.parametrize("scheme,order", [("LAD_C6", 6.0), ("LAD_E4", 4.0)])
def test_metric_convergence_order(scheme, order):
    errs = []
    for n in (16, 32):
        xyz, per = inputs.wavy_grid_2d(n, n, amp=0.05)
        prob = inputs.uniform_flow_curvilinear(xyz, per, (1.0, 0.3, 0.2, 1.0))
        node, _ = oracle.Oracle(prob, scheme=scheme).metrics()
        exact = _analytic_wavy_2d(n, n, 0.05)
        # relative to the metric scale 1/n
        errs.append(float(np.abs(node[:4] - exact).max()) * n)
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - order) <= 0.35, (scheme, errs, rate)


def test_freestream_on_a_small_compression_ramp_grid():
    """The ramp's body-fitted grid (stretched, cornered, spanwise periodic),
    downsized: a uniform stream stays uniform under LAD-C6 (inviscid and
    viscous), as under LAD-E4."""
    ramp = inputs.compression_ramp(nx=40, ny=24, nz=8)
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
    for viscous in (False, True):
        p = inputs._viscous(dict(prob), 2400.0, 2.9, ramp["suth"], ramp["t_wall"]) if viscous else prob
        for scheme in ("LAD_E4", "LAD_C6"):
            o = oracle.Oracle(p, scheme=scheme)
            R = o.rhs(p["U"])
            J = o.metrics()[0][-1]
            assert np.abs(R / J).max() <= 1e-11 * np.abs(p["U"]).max(), (scheme, viscous)


def test_conservation_3d_wavy_with_filter():
    """Periodic 3D wavy grid: sum(Q/J) is conserved to round-off over four
    LAD-C6 steps, filter included."""
    xyz, per = inputs.wavy_grid_3d((12, 10, 8), amp=0.05)
    x, y, z = xyz
    W = np.stack([1.0 + 0.2 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * z), 0.4 + 0 * x,
                  0.1 * np.cos(2 * math.pi * y), -0.2 + 0 * x, 1.0 + 0.1 * np.sin(2 * math.pi * (x + y))])
    prob = inputs.field_on_curvilinear(xyz, per, W)
    o = oracle.Oracle(prob, scheme="LAD_C6", cfl=0.1)
    J = o.metrics()[0][-1]
    U, _, _ = o.advance(prob["U"], nsteps=4)
    assert not np.array_equal(U, prob["U"])
    for v in range(5):
        a, b = (prob["U"][v] / J).sum(), (U[v] / J).sum()
        assert abs(a - b) <= 1e-13 * np.abs(prob["U"][v] / J).sum(), v


def test_filter_conserves_q_over_j_and_keeps_cartesian_arithmetic():
    """On a curvilinear periodic grid the filter alone keeps sum(Q/J) (not
    sum(Q)); on a uniform grid it is the plain filter of Q."""
    xyz, per = inputs.wavy_grid_2d(24, 20, amp=0.08)
    x, y = xyz
    W = np.stack([1.0 + 0.3 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y), 0.5 + 0 * x,
                  0.2 + 0.1 * np.cos(2 * math.pi * y), 1.0 + 0.2 * np.sin(2 * math.pi * (x + y))])
    prob = inputs.field_on_curvilinear(xyz, per, W)
    o = oracle.Oracle(prob, scheme="LAD_C6")
    J = o.metrics()[0][-1]
    Uf = o.filter(prob["U"])
    for v in range(4):
        assert abs((Uf[v] / J).sum() - (prob["U"][v] / J).sum()) <= 1e-14 * np.abs(prob["U"][v] / J).sum()
    kh = inputs.kelvin_helmholtz(32)
    Ukh = oracle.Oracle(kh, scheme="LAD_C6").filter(kh["U"])
    for v in range(4):  # periodic lines: the plain filter keeps sum(Q)
        assert abs(Ukh[v].sum() - kh["U"][v].sum()) <= 1e-13 * np.abs(kh["U"][v]).sum()
