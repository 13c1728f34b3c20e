"""Pins of the C-GBR reconstruction, the reflective wall and the per-interface
hybrid mask of the FP64 oracle, against properties the paper and the
mathematics fix (CPU only):

* Eq. (7)-(8): below the thresholds the entropy and shear waves take the
  centralised state, the average of the two one-sided linear states.  That
  average is symmetric about the interface, so the semi-discrete operator of a
  small entropy or shear wave is skew-symmetric: the wave's discrete energy
  sum(w'^2) does not change.  An upwind state makes it decay, as the acoustic
  waves do.
* Sec. 2.3: the characteristic frame is the eigenbasis of the primitive
  Euler Jacobian at the arithmetic mean of the two interface nodes.
* Sec. 2.1 boundary treatment: a reflective slip wall is the mirror plane of a
  periodic flow on the doubled domain (u odd, rho, v, p even).
* Sec. 5: in the per-interface hybrid, exactly the interfaces with a troubled
  node on either side carry the C-GBR (MEG6) flux; every other interface
  carries the LAD-E4 flux form.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_18042_gb300 import inputs

G = 1.4


def _x_wave(n, rho, u, v, p, ny=4):
    """2D periodic grid (n x ny) whose state varies along x only."""
    h = 1.0 / n
    W = np.stack([rho, u, v, p])
    W = np.ascontiguousarray(np.broadcast_to(W[:, None, :], (4, ny, n)))
    return inputs._problem("xwave", 2, [n, ny], [h, h], [[0, 0], [0, 0]], W, G)


def _profile(n):
    x = (np.arange(n) + 0.5) / n
    return np.sin(2 * math.pi * x) + 0.5 * np.cos(4 * math.pi * x + 0.3)


def _energy_rate(pert, rate):
    """sum(w' dw'/dt) normalised by |w'| |dw'/dt|: zero for a skew-symmetric
    (non-dissipative) operator, negative for a dissipative one."""
    return float(np.dot(pert, rate) / (np.linalg.norm(pert) * np.linalg.norm(rate)))


# ------------------------------------------------------------ Eq. (7)-(8) centralised states
@pytest.mark.parametrize("n", [8, 16])
@pytest.mark.parametrize("u0", [0.7, -0.6])
def test_shear_wave_takes_the_central_state(n, u0):
    """A shear wave v = eps s(x) advected by u0 at rest pressure and density:
    Omega^d vanishes (no pressure variation, no dilatation), so the shear
    characteristic takes the central state (Eq. 8, b = 3, 4) and the discrete
    energy of v is conserved to round-off, for either flow direction."""
    one = np.ones(n)
    eps = 1e-3 * _profile(n)
    prob = _x_wave(n, one, u0 * one, eps, one)
    R = oracle.Oracle(prob, scheme="MEG6").rhs(prob["U"])
    assert np.abs(R[0]).max() <= 1e-14  # mass flux rho * u0 is uniform
    assert abs(_energy_rate(eps, R[2, 1])) <= 1e-12


@pytest.mark.parametrize("n", [8, 16])
@pytest.mark.parametrize("u0", [0.7, -0.6])
def test_entropy_wave_takes_the_central_state(n, u0):
    """A density wave at uniform u0 and p: with the MP tolerance of Eq. (8)
    raised to 1 the entropy criterion selects the central linear state at
    every interface, and the discrete energy of the density perturbation is
    conserved to round-off.  With the printed tolerance (1e-20) and an
    amplitude small enough that the linear state stays inside it, the same
    holds to the rounding of R at that amplitude."""
    one = np.ones(n)
    s = _profile(n)
    prob = _x_wave(n, one + 1e-3 * s, u0 * one, 0 * one, one)
    R = oracle.Oracle(prob, scheme="MEG6", mp_eps=1.0).rhs(prob["U"])
    assert abs(_energy_rate(s, R[0, 1])) <= 1e-11
    prob = _x_wave(n, one + 1e-11 * s, u0 * one, 0 * one, one)
    R = oracle.Oracle(prob, scheme="MEG6").rhs(prob["U"])
    assert abs(_energy_rate(s, R[0, 1])) <= 5e-5


@pytest.mark.parametrize("n", [8, 16])
def test_acoustic_wave_takes_the_upwind_state(n):
    """The contrast that shows the measure has teeth: a small right-running
    acoustic wave (dp = rho c du, drho = dp / c^2) takes the upwind linear
    states (Eq. 8, b = 1, 5, below the sensor threshold) and loses energy."""
    one = np.ones(n)
    c = math.sqrt(G)
    dp = 1e-5 * _profile(n)
    prob = _x_wave(n, one + dp / c ** 2, dp / c, 0 * one, one + dp)
    o = oracle.Oracle(prob, scheme="MEG6")
    assert o.omega(prob["U"]).max() < 0.01
    R = o.rhs(prob["U"])
    assert _energy_rate(dp, R[3, 1]) < -1e-4


# ------------------------------------------------------------ Sec. 2.3 characteristic frame
def _primitive_jacobian(W, nvec):
    """A_n of the primitive Euler system W_t + A_n W_n = 0 (rho, u, p)."""
    nd = len(nvec)
    rho, u, p = W[0], np.asarray(W[1:1 + nd]), W[1 + nd]
    un = float(np.dot(u, nvec))
    c2 = G * p / rho
    A = np.zeros((nd + 2, nd + 2))
    A[0, 0] = un
    A[0, 1:1 + nd] = rho * nvec
    for k in range(nd):
        A[1 + k, 1 + k] = un
        A[1 + k, 1 + nd] = nvec[k] / rho
    A[1 + nd, 1:1 + nd] = rho * c2 * nvec
    A[1 + nd, 1 + nd] = un
    return A


@pytest.mark.parametrize("nd", [1, 2, 3])
def test_frame_is_the_eigenbasis_at_the_mean_state(nd):
    rng = np.random.default_rng(7 + nd)
    for _ in range(50):
        Wi = np.concatenate([[rng.uniform(0.1, 3)], rng.uniform(-2, 2, nd), [rng.uniform(0.1, 3)]])
        Wj = np.concatenate([[rng.uniform(0.1, 3)], rng.uniform(-2, 2, nd), [rng.uniform(0.1, 3)]])
        xi = rng.uniform(-2, 2, nd)
        xi[0] += 2.5 * np.sign(xi[0] + 1e-300)
        I = np.eye(nd + 2)
        L = np.stack([oracle.char_transform(Wi, Wj, xi, I[k]) for k in range(nd + 2)], axis=1)
        Rm = np.stack([oracle.char_transform(Wi, Wj, xi, I[k], inverse=True) for k in range(nd + 2)], axis=1)
        assert np.abs(Rm @ L - I).max() <= 1e-13
        nvec = xi / np.linalg.norm(xi)
        Wm = 0.5 * (Wi + Wj)
        c = math.sqrt(G * Wm[-1] / Wm[0])
        un = float(np.dot(Wm[1:1 + nd], nvec))
        D = L @ _primitive_jacobian(Wm, nvec) @ Rm
        want = np.diag([un - c] + [un] * nd + [un + c])
        assert np.abs(D - want).max() <= 1e-12 * (abs(un) + c)
        # a right-running acoustic jump of the mean state is carried by the last wave alone
        dp = 0.37
        dW = np.concatenate([[dp / c ** 2], dp / (Wm[0] * c) * nvec, [dp]])
        cv = oracle.char_transform(Wi, Wj, xi, dW)
        assert np.abs(cv[:-1]).max() <= 1e-14 and abs(cv[-1] - dp / c ** 2) <= 1e-14


# ------------------------------------------------------------ Sec. 2.1 reflective slip wall
def _wall_state(X, Y, Ly):
    """A smooth state with no symmetry of its own, periodic in y."""
    cy, sy = np.cos(2 * math.pi * Y / Ly), np.sin(2 * math.pi * Y / Ly)
    rho = 1.0 + 0.2 * np.cos(2.0 * X) + 0.05 * cy * X
    u = 0.3 * np.sin(3.0 * X + 0.4) * (1.0 + 0.2 * sy)
    v = 0.2 + 0.1 * np.cos(2.5 * X) * cy
    p = 1.0 + 0.1 * np.cos(1.7 * X + 0.2) + 0.05 * sy * X
    return np.stack([rho, u, v, p])


@pytest.mark.parametrize("scheme,kw", [("MEG6", {}), ("LAD_E4", {}),
                                       ("HYBRID", dict(hybrid_mode=1, hyb_rho=1.0))])
def test_reflective_wall_is_the_mirror_of_the_doubled_domain(scheme, kw):
    """Reflective walls at x = 0 and x = L (mirror about the boundary face,
    wall-normal velocity negated) against the periodic domain [-L, L] holding
    the state and its mirror image (u negated, rho, v, p kept): the
    right-hand sides agree on [0, L]."""
    nx, ny = 20, 12
    L, Ly = 1.0, 0.6
    h = L / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * (Ly / ny)
    X, Y = np.meshgrid(x, y)
    W = _wall_state(X, Y, Ly)
    wall = inputs._problem("wall", 2, [nx, ny], [h, Ly / ny], [[2, 2], [0, 0]], W, G)
    Wm = W[:, :, ::-1].copy()
    Wm[1] = -Wm[1]
    per = inputs._problem("doubled", 2, [2 * nx, ny], [h, Ly / ny], [[0, 0], [0, 0]],
                          np.concatenate([Wm, W], axis=2), G)
    Rw = oracle.Oracle(wall, scheme=scheme, **kw).rhs(wall["U"])
    Rp = oracle.Oracle(per, scheme=scheme, **kw).rhs(per["U"])[:, :, nx:]
    for v in range(4):
        assert np.abs(Rw[v] - Rp[v]).max() <= 1e-12 * np.abs(Rp).max(), v


# ------------------------------------------------------------ Sec. 5 per-interface mask
@pytest.mark.parametrize("buf", [0, 1])
def test_per_interface_mask_marks_both_interfaces_of_a_troubled_node(buf):
    """buf = 0: the rule as read.  buf = 1: the troubled node also marks its
    eight neighbours, so the 3 x 3 block's interfaces take the C-GBR flux."""
    nx, ny = 24, 16
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * (1.0 / ny)
    X, Y = np.meshgrid(x, y)
    W = np.stack([1.0 + 0.1 * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y),
                  0.3 + 0.1 * np.cos(2 * math.pi * Y), -0.2 + 0.1 * np.sin(2 * math.pi * X),
                  1.0 + 0.05 * np.cos(2 * math.pi * (X + Y))])
    i0, j0 = 11, 7
    W[0, j0, i0] = 0.3  # the one troubled node: rho below the threshold 0.5
    prob = inputs._problem("mask", 2, [nx, ny], [h, 1.0 / ny], [[0, 0], [0, 0]], W, G)
    U = prob["U"]
    hyb = oracle.Oracle(prob, scheme="HYBRID", hybrid_mode=1, hyb_rho=0.5, hybrid_buffer=buf)
    none = oracle.Oracle(prob, scheme="HYBRID", hybrid_mode=1)  # no node troubled: LAD-E4 flux form
    meg = oracle.Oracle(prob, scheme="MEG6")
    assert hyb.hybrid_flag(U) == 1
    for d, (line, node) in enumerate(((j0, i0), (i0, j0))):
        Fh, Fn, Fm = hyb.iface_flux(U, d), none.iface_flux(U, d), meg.iface_flux(U, d)
        mask = np.zeros(Fh.shape[1:], dtype=bool)
        # interfaces node - 1/2 - buf .. node + 1/2 + buf of lines line - buf .. line + buf
        mask[line - buf:line + buf + 1, node - buf:node + buf + 2] = True
        assert np.array_equal(Fh[:, mask], Fm[:, mask]), d
        assert np.array_equal(Fh[:, ~mask], Fn[:, ~mask]), d
        # the two fluxes differ at the marked interfaces, so the pin is not vacuous
        assert np.abs(Fm[:, mask] - Fn[:, mask]).max() > 1e-4 * np.abs(Fm).max(), d


# ------------------------------------------------------------ Sec. 5 robustness of the buffer
def test_buffer_keeps_an_expanding_vortex_sheet_positive():
    """Quadrant Riemann problem 152 of the seeded batch (75 x 75): the bottom
    quadrants separate (du = 1.26) along a vortex sheet (dv = 1.29) without a
    pressure jump, so Omega never flags it.  LAD-E4 has no artificial shear
    viscosity and drains the density there; the per-interface hybrid with the
    rule as read (buffer 0) goes non-physical by step 30, MEG6 alone and the
    hybrid with a one-node buffer stay positive."""
    p = inputs.batched_riemann(count=256, seed=0)[152]
    st = p["quad_states"]
    kw = dict(scheme="HYBRID", hybrid_mode=1, hybrid_sensor=1, hyb_rho=0.5 * float(st[:, 0].min()),
              hyb_p=0.5 * float(st[:, 3].min()))

    def positive_after(o, steps):
        U = p["U"]
        for _ in range(steps):
            U = o.rk3_step(U, o.cfl_dt(U))
            pr = 0.4 * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
            if not (np.isfinite(U).all() and U[0].min() > 0 and pr.min() > 0):
                return False
        return True

    assert not positive_after(oracle.Oracle(p, **kw), 30)
    assert positive_after(oracle.Oracle(p, hybrid_buffer=1, **kw), 40)
    assert positive_after(oracle.Oracle(p, scheme="MEG6"), 40)
