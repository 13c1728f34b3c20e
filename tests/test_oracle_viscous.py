"""Pins of the oracle's physical viscous terms (Sec. 2.1, Eq. 3: Newtonian
stress with Stokes' hypothesis, Fourier conduction kappa_hat = mu_hat /
((gamma-1) Pr M^2), Sutherland viscosity), the isothermal no-slip wall and the
per-node inflow profile, against closed forms, symmetry and convergence:

* a periodic shear wave and a wall-bounded one decay at the discrete rate
  nu k*^2, with k* the modified wavenumber of the central derivative used
  twice (E4 or C6), and the energy source equals the closed form of
  d/dy (u tau_xy);
* with odd velocity and temperature deviation, the no-slip isothermal wall
  is the mirror of a periodic flow on the doubled channel: the right-hand
  sides agree on the upper half;
* in 3D, Cartesian and curvilinear, the viscous part of the right-hand side
  converges at fourth order to mu (lap u + grad(div u)/3) and
  u . div(tau) + tau : grad(u);
* heat conduction at rest converges to d/dx (kappa(T) dT/dx);
* a parallel shear flow fed by its own inflow profile is steady;
* Sutherland's law against the tabulated viscosity of air.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_18042_gb300 import inputs

GAMMA = 1.4


def kstar_e4(k, h):
    return (8.0 * math.sin(k * h) - math.sin(2 * k * h)) / (6.0 * h)


def kstar_c6(k, h):
    return ((14.0 / 9.0) * math.sin(k * h) + (1.0 / 18.0) * math.sin(2 * k * h)) / (
        (1.0 + (2.0 / 3.0) * math.cos(k * h)) * h)


def mu_hat(p):
    return 1.0 / p["re"]  # T = 1 in these cases


@pytest.mark.parametrize("scheme,ks", [("MEG6", kstar_e4), ("MIG4", kstar_e4), ("LAD_E4", kstar_e4),
                                       ("LAD_C6", kstar_c6), ("HYBRID", kstar_e4)])
def test_shear_wave_discrete_decay_rate(scheme, ks):
    n = 32
    p = inputs.shear_wave(n=n, amp=1e-3, minf=0.2, re=100.0)
    kw = dict(hybrid_mode=oracle.HYB_CELL, hyb_rho=0.5) if scheme == "HYBRID" else {}
    o = oracle.Oracle(p, scheme=scheme, **kw)
    R = o.rhs(p["U"])
    h = 1.0 / n
    k = 2 * math.pi
    kk = ks(k, h)
    mu = mu_hat(p)
    U = p["U"]
    scale = mu * kk * kk * 1e-3
    assert np.abs(R[1] - (-mu * kk * kk) * U[1]).max() <= 1e-12 * scale
    assert np.abs(R[0]).max() <= 1e-12 * scale and np.abs(R[2]).max() <= 1e-12 * scale
    y = (np.arange(n) + 0.5) * h
    Ry = 0.5 * mu * 1e-6 * kk * ks(2 * k, h) * np.cos(2 * k * y)
    assert np.abs(R[3] - Ry[:, None]).max() <= 1e-9 * np.abs(Ry).max()


@pytest.mark.parametrize("scheme", ["MEG6", "LAD_E4"])
def test_wall_bounded_shear_decays_like_the_doubled_sine(scheme):
    n = 32
    p = inputs.wall_channel(n=n, nx=8, minf=0.5, re=50.0, suth=0.5, twall=1.0)
    o = oracle.Oracle(p, scheme=scheme)
    R = o.rhs(p["U"])
    kk = kstar_e4(math.pi, 1.0 / n)
    mu = 1.0 / 50.0
    ref = (-mu * kk * kk) * p["U"][1]
    assert np.abs(R[1] - ref).max() <= 1e-11 * np.abs(ref).max()


def _odd_even_fields(Lx, tw, p0):
    def f(X, Y):
        u = 0.02 * np.sin(math.pi * Y) * (1.0 + 0.3 * np.cos(2 * math.pi * X / Lx))
        v = 0.01 * np.sin(2 * math.pi * Y) * np.sin(2 * math.pi * X / Lx)
        p = p0 * (1.0 + 0.05 * np.cos(math.pi * Y))
        T = tw + 0.1 * np.sin(math.pi * Y) * (1.0 + 0.2 * np.cos(2 * math.pi * X / Lx))
        return u, v, p, T
    return f


def test_wall_is_the_mirror_of_the_doubled_periodic_channel():
    n, nx, minf, tw = 16, 8, 0.5, 1.3
    p0 = 1.0 / (GAMMA * minf * minf)
    Lx = nx / n
    f = _odd_even_fields(Lx, tw, p0)
    wall = inputs.wall_channel(n=n, nx=nx, minf=minf, re=40.0, suth=0.6, twall=tw, fields=f)
    # the same fields on [-1, 1], periodic in y, 2n rows
    h = 1.0 / n
    x = (np.arange(nx) + 0.5) * h
    y = -1.0 + (np.arange(2 * n) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    u, v, pp, T = f(X, Y)
    W = np.stack([GAMMA * minf * minf * pp / T, u, v, pp])
    per = inputs._problem("doubled", 2, [nx, 2 * n], [h, h], [[0, 0], [0, 0]], W, GAMMA)
    per = inputs._viscous(per, 40.0, minf, 0.6, tw)
    Rw = oracle.Oracle(wall, scheme="MEG6").rhs(wall["U"])
    Rp = oracle.Oracle(per, scheme="MEG6").rhs(per["U"])[:, n:, :]
    for v in range(4):
        assert np.abs(Rw[v] - Rp[v]).max() <= 1e-10 * np.abs(Rp[v]).max(), v


def _field3(P):
    """Smooth periodic velocity (div != 0), rho = 1, uniform p -> T = 1."""
    x, y, z = P
    tp = 2 * math.pi
    u = np.stack([0.1 * np.sin(tp * x) + 0.05 * np.sin(tp * y),
                  0.08 * np.sin(tp * y) + 0.04 * np.cos(tp * z),
                  0.06 * np.sin(tp * z) + 0.03 * np.sin(tp * x)])
    # velocity gradient G[i][j] = du_i / dx_j
    G = np.zeros((3, 3) + x.shape)
    G[0, 0] = 0.1 * tp * np.cos(tp * x)
    G[0, 1] = 0.05 * tp * np.cos(tp * y)
    G[1, 1] = 0.08 * tp * np.cos(tp * y)
    G[1, 2] = -0.04 * tp * np.sin(tp * z)
    G[2, 2] = 0.06 * tp * np.cos(tp * z)
    G[2, 0] = 0.03 * tp * np.cos(tp * x)
    lap = np.stack([-(tp ** 2) * (0.1 * np.sin(tp * x) + 0.05 * np.sin(tp * y)),
                    -(tp ** 2) * (0.08 * np.sin(tp * y) + 0.04 * np.cos(tp * z)),
                    -(tp ** 2) * (0.06 * np.sin(tp * z) + 0.03 * np.sin(tp * x))])
    graddiv = np.stack([-0.1 * tp * tp * np.sin(tp * x), -0.08 * tp * tp * np.sin(tp * y),
                        -0.06 * tp * tp * np.sin(tp * z)])
    return u, G, lap, graddiv


def _visc_error(n, curvilinear, scheme):
    minf, re = 0.3, 20.0
    mu = 1.0 / re
    if curvilinear:
        xyz, per = inputs.wavy_grid_3d((n, n, n), amp=0.05)
        P = xyz
    else:
        h = 1.0 / n
        c = (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        P = np.stack([X, Y, Z])
    u, G, lap, graddiv = _field3(P)
    p0 = 1.0 / (GAMMA * minf * minf)
    W = np.concatenate([np.ones((1,) + P.shape[1:]), u, np.full((1,) + P.shape[1:], p0)])
    if curvilinear:
        prob = inputs.field_on_curvilinear(xyz, per, W)
    else:
        prob = inputs._problem("box", 3, [n] * 3, [1.0 / n] * 3, [[0, 0]] * 3, W, GAMMA)
    inv = dict(prob)
    vis = inputs._viscous(dict(prob), re, minf, 0.0, 1.0)
    inv.update(minf=minf)
    Rv = oracle.Oracle(vis, scheme=scheme).rhs(vis["U"])
    Ri = oracle.Oracle(inv, scheme=scheme).rhs(inv["U"])
    D = Rv - Ri
    divt = mu * (lap + graddiv / 3.0)
    div = G[0, 0] + G[1, 1] + G[2, 2]
    tau = np.empty((3, 3) + div.shape)
    for i in range(3):
        for j in range(3):
            tau[i, j] = mu * (G[i, j] + G[j, i]) - (i == j) * (2.0 / 3.0) * mu * div
    work = sum(u[i] * divt[i] for i in range(3)) + sum(tau[i, j] * G[i, j] for i in range(3) for j in range(3))
    err_m = max(np.abs(D[1 + i] - divt[i]).max() for i in range(3))
    err_e = np.abs(D[4] - work).max()
    return err_m / np.abs(divt).max(), err_e / np.abs(work).max(), np.abs(D[0]).max()


@pytest.mark.parametrize("curv", [False, True])
@pytest.mark.parametrize("scheme", ["MEG6", "LAD_E4"])
def test_3d_viscous_terms_converge_at_fourth_order(curv, scheme):
    e1m, e1e, m1 = _visc_error(12, curv, scheme)
    e2m, e2e, m2 = _visc_error(24, curv, scheme)
    assert m1 <= 1e-12 and m2 <= 1e-12  # no viscous mass flux
    assert e2m < 0.02 and e2e < 0.02
    assert e1m / e2m > 10.0 and e1e / e2e > 10.0, (e1m / e2m, e1e / e2e)


def _heat_error(n, suth):
    minf, re, a = 0.4, 30.0, 0.3
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    T = 1.0 + a * np.sin(2 * math.pi * x)
    p0 = 1.0 / (GAMMA * minf * minf)
    W = np.stack([GAMMA * minf * minf * p0 / T, 0 * x, np.full(n, p0)])
    prob = inputs._viscous(inputs._problem("heat", 1, [n], [h], [[0, 0]], W, GAMMA), re, minf, suth, 1.0)
    R = oracle.Oracle(prob, scheme="MEG6").rhs(prob["U"])
    mu = T ** 1.5 * (1 + suth) / (T + suth) / re
    dmu = mu * (1.5 / T - 1.0 / (T + suth))
    kc = (GAMMA - 1.0) * 0.72 * minf * minf
    Tx = a * 2 * math.pi * np.cos(2 * math.pi * x)
    Txx = -a * (2 * math.pi) ** 2 * np.sin(2 * math.pi * x)
    ref = (dmu * Tx * Tx + mu * Txx) / kc
    return np.abs(R[2] - ref).max() / np.abs(ref).max(), np.abs(R[0]).max() + np.abs(R[1]).max()


def test_heat_conduction_at_rest_converges_to_the_conduction_term():
    e1, z1 = _heat_error(32, 0.5)
    e2, z2 = _heat_error(64, 0.5)
    assert z1 <= 1e-12 and z2 <= 1e-12
    assert e2 < 1e-3 and e1 / e2 > 12.0


@pytest.mark.parametrize("scheme", ["MEG6", "LAD_E4"])
def test_parallel_shear_flow_fed_by_its_own_inflow_profile_is_steady(scheme):
    nx, ny, nz = 10, 8, 6
    h = 0.1
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Zg, Yg, Xg = np.meshgrid(z, y, np.arange(nx), indexing="ij")
    W = np.zeros((5, nz, ny, nx))
    W[0] = 1.0  # uniform e: no artificial conduction (LAD)
    W[1] = 1.5 + 0.3 * np.sin(2 * math.pi * Yg) + 0.1 * np.cos(2 * math.pi * Zg)
    W[4] = 0.7
    prob = inputs._problem("parallel", 3, [nx, ny, nz], [h, 1.0 / ny, 1.0 / nz],
                           [[inputs.INFLOW, inputs.EXTRAP], [0, 0], [0, 0]], W, GAMMA)
    prof = np.ascontiguousarray(W[:, :, :, 0].reshape(5, -1))
    prob["inflow"] = {(0, 0): (1.0, 1.0, 0.0, 0.0, 0.7)}
    prob["inflow_profile"] = {(0, 0): prof}
    R = oracle.Oracle(prob, scheme=scheme).rhs(prob["U"])
    assert np.abs(R).max() <= 1e-12 * np.abs(prob["U"]).max() / h
    # control: the profile transposed in (y, z) is not the flow's own profile
    bad = dict(prob)
    bad["inflow_profile"] = {(0, 0): np.ascontiguousarray(
        W[:, :, :, 0].transpose(0, 2, 1)[:, :ny, :nz].reshape(5, -1)[:, :ny * nz])}
    Rb = oracle.Oracle(bad, scheme=scheme).rhs(prob["U"])
    assert np.abs(Rb).max() > 1e-3


def test_sutherland_law_matches_tabulated_air_viscosity():
    """mu(300 K) / mu(273.15 K) of air = 1.846e-5 / 1.716e-5 (White, Viscous
    Fluid Flow, Table 1-2 / Sutherland constants 273.15 K, 110.4 K)."""
    t0 = 273.15
    ratio_tab = 1.846 / 1.716
    n = 32
    T = 300.0 / t0
    minf = 0.2
    p = inputs.shear_wave(n=n, amp=1e-3, minf=minf, re=100.0, suth=110.4 / t0)
    # uniform temperature T: rho = 1, p = rho T / (gamma M^2)
    U = p["U"].copy()
    pr = T / (GAMMA * minf * minf)
    U[3] = pr / (GAMMA - 1.0) + 0.5 * U[1] * U[1] / U[0]
    R = oracle.Oracle(p, scheme="LAD_E4").rhs(U)
    kk = kstar_e4(2 * math.pi, 1.0 / n)
    mu_eff = -R[1] / (kk * kk * U[1])
    ratio = float(np.median(mu_eff)) * 100.0
    assert abs(ratio - ratio_tab) <= 2e-3 * ratio_tab
