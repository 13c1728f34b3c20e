"""Seeded synthetic problem setups (initial data only).

Shared by the tests, the benchmark and the CPU baseline.  It holds no step of
the numerical method: it lays out grids, boundary types and initial states and
forms the conserved variables of an ideal gas from primitive initial data
(rho, rho*u, E = p/(gamma-1) + rho|u|^2/2, energy per unit volume).

Every problem is a dict:
  name, ndim, n (3 ints), h (3 spacings), bc (ndim x 2 boundary types),
  inflow {(dir, side): primitive state}, gamma, U (nv, [nz,] [ny,] nx) FP64,
  optionally xyz (ndim, [nz,] [ny,] nx) node coordinates and period
  (ndim x ndim translations across periodic directions), t_end, cfl.
Node positions are cell centres x_i = lo + (i + 1/2) h.
"""
import math

import numpy as np

PERIODIC, EXTRAP, REFLECT, INFLOW = 0, 1, 2, 3


def prim_to_cons(W, gamma):
    """W: (ndim+2, ...) primitive (rho, u.., p) -> conserved."""
    nd = W.shape[0] - 2
    U = np.empty_like(W)
    rho = W[0]
    U[0] = rho
    q = np.zeros_like(rho)
    for k in range(nd):
        U[1 + k] = rho * W[1 + k]
        q = q + W[1 + k] * W[1 + k]
    U[nd + 1] = W[nd + 1] / (gamma - 1.0) + 0.5 * rho * q
    return U


def _problem(name, ndim, n, h, bc, W, gamma, **kw):
    n3 = list(n) + [1] * (3 - len(n))
    h3 = list(h) + [1.0] * (3 - len(h))
    d = dict(name=name, ndim=ndim, n=n3, h=h3, bc=[list(b) for b in bc], gamma=gamma,
             U=np.ascontiguousarray(prim_to_cons(W, gamma)), inflow={})
    d.update(kw)
    return d


SHOCK_TUBES = {
    # (left state, right state, x0, domain length, t_end, gamma); Sec. 3.1
    "sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 0.5, 1.0, 0.2, 1.4),
    "lax": ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571), 0.5, 1.0, 0.14, 1.4),
    "leblanc": ((1.0, 0.0, 2.0 / 3.0 * 1e-1), (1e-3, 0.0, 2.0 / 3.0 * 1e-10), 3.0, 9.0, 6.0, 5.0 / 3.0),
}


def shock_tube(name="sod", N=400, cfl=0.5):
    WL, WR, x0, L, t_end, gamma = SHOCK_TUBES[name]
    h = L / N
    x = (np.arange(N) + 0.5) * h
    W = np.empty((3, N))
    left = x < x0
    for v in range(3):
        W[v] = np.where(left, WL[v], WR[v])
    p = _problem(name, 1, [N], [h], [[INFLOW, EXTRAP]], W, gamma, t_end=t_end, cfl=cfl,
                 x=x, x0=x0, WL=WL, WR=WR)
    p["inflow"] = {(0, 0): WL}
    return p


def triple_point(nx=1792, ny=768, cfl=0.2):
    """Triple point (Sec. 3.2), [0,7]x[0,3], reflective walls, gamma 1.4."""
    hx, hy = 7.0 / nx, 3.0 / ny
    x = (np.arange(nx) + 0.5) * hx
    y = (np.arange(ny) + 0.5) * hy
    X, Y = np.meshgrid(x, y)
    W = np.zeros((4, ny, nx))
    W[0] = np.where(X < 1.0, 1.0, np.where(Y < 1.5, 1.0, 0.125))
    W[3] = np.where(X < 1.0, 1.0, 0.1)
    return _problem("triple_point", 2, [nx, ny], [hx, hy], [[REFLECT, REFLECT], [REFLECT, REFLECT]],
                    W, 1.4, t_end=3.5, cfl=cfl, rho_c3=0.125)


def riemann_c3(n=64, cfl=0.2):
    """Strong 2D Riemann problem, configuration 3 (Sec. 3.2); extrapolation walls."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    s = 4.0 / math.sqrt(11.0)
    q = {  # (rho, u, v, p)
        "ne": (1.5, 0.0, 0.0, 1.5), "nw": (33.0 / 62.0, s, 0.0, 0.3),
        "sw": (77.0 / 558.0, s, s, 9.0 / 310.0), "se": (33.0 / 62.0, 0.0, s, 0.3),
    }
    W = np.zeros((4, n, n))
    east, north = X > 0.8, Y > 0.8
    for v in range(4):
        W[v] = np.where(north, np.where(east, q["ne"][v], q["nw"][v]),
                        np.where(east, q["se"][v], q["sw"][v]))
    return _problem("riemann_c3", 2, [n, n], [h, h], [[EXTRAP, EXTRAP], [EXTRAP, EXTRAP]], W, 1.4,
                    t_end=0.8, cfl=cfl)


def kelvin_helmholtz(n=64, cfl=0.2):
    """Periodic Kelvin-Helmholtz setup (Sec. 3.2) on [0,1]^2."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    band = (Y > 0.25) & (Y <= 0.75)
    sig = 0.05 / math.sqrt(2.0)
    W = np.zeros((4, n, n))
    W[0] = np.where(band, 2.0, 1.0)
    W[1] = np.where(band, 0.5, -0.5)
    W[2] = 0.1 * np.sin(4 * math.pi * X) * (np.exp(-(Y - 0.75) ** 2 / (2 * sig * sig)) +
                                            np.exp(-(Y - 0.25) ** 2 / (2 * sig * sig)))
    W[3] = 2.5
    return _problem("kelvin_helmholtz", 2, [n, n], [h, h], [[PERIODIC, PERIODIC]] * 2, W, 1.4,
                    t_end=0.8, cfl=cfl)


def entropy_wave(ndim=1, n=64, amp=0.2, direction=0):
    """Smooth periodic entropy wave rho = 1 + amp sin(2 pi x_d), u_d = 1, p = 1 on [0,1]^ndim."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    grids = np.meshgrid(*([x] * ndim), indexing="ij")[::-1] if ndim > 1 else [x]
    # grids[k] varies along array axis (ndim-1-k) ... build explicitly instead
    shape = (n,) * ndim
    coords = []
    for d in range(ndim):
        sh = [1] * ndim
        sh[ndim - 1 - d] = n
        coords.append(np.broadcast_to(x.reshape(sh), shape))
    W = np.zeros((ndim + 2,) + shape)
    W[0] = 1.0 + amp * np.sin(2 * math.pi * coords[direction])
    W[1 + direction] = 1.0
    W[ndim + 1] = 1.0
    del grids
    return _problem("entropy_wave", ndim, [n] * ndim, [h] * ndim, [[PERIODIC, PERIODIC]] * ndim, W,
                    1.4, amp=amp, direction=direction)


def random_quadrants(rng, n):
    """One 2D quadrant Riemann problem (batched / serving mixes): unit square,
    seeded centre, rho~U[0.1,2], p~U[0.05,1.5], u,v~U[-1,1]; transmissive walls."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    x0, y0 = rng.uniform(0.0, 1.0, size=2)
    st = np.stack([rng.uniform(0.1, 2.0, 4), rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 4),
                   rng.uniform(0.05, 1.5, 4)], axis=1)
    quad = np.where(Y > y0, np.where(X > x0, 0, 1), np.where(X > x0, 3, 2))
    W = np.empty((4, n, n))
    for v in range(4):
        W[v] = st[quad, v]
    return _problem("quadrants", 2, [n, n], [h, h], [[EXTRAP, EXTRAP], [EXTRAP, EXTRAP]], W, 1.4,
                    cfl=0.2, quad_states=st, centre=(x0, y0))


def random_tube(rng, N):
    """One 1D shock tube of the serving mix: rho, p ~ U[0.1,2], u ~ U[-1,1] per side."""
    h = 1.0 / N
    x = (np.arange(N) + 0.5) * h
    WL = (rng.uniform(0.1, 2.0), rng.uniform(-1, 1), rng.uniform(0.1, 2.0))
    WR = (rng.uniform(0.1, 2.0), rng.uniform(-1, 1), rng.uniform(0.1, 2.0))
    W = np.empty((3, N))
    for v in range(3):
        W[v] = np.where(x < 0.5, WL[v], WR[v])
    return _problem("tube", 1, [N], [h], [[EXTRAP, EXTRAP]], W, 1.4, cfl=0.5, WL=WL, WR=WR)


def wavy_grid_2d(nx=32, ny=32, amp=0.1, Lx=1.0, Ly=1.0):
    """Sinusoidally perturbed periodic curvilinear grid (freestream tests)."""
    i = np.arange(nx)
    j = np.arange(ny)
    I, J = np.meshgrid(i, j)
    xs, ys = I / nx, J / ny
    x = Lx * (xs + amp * np.sin(2 * math.pi * xs) * np.sin(2 * math.pi * ys))
    y = Ly * (ys + amp * np.sin(2 * math.pi * xs) * np.sin(2 * math.pi * ys))
    return np.stack([x, y]), [[Lx, 0.0], [0.0, Ly]]


def wavy_grid_3d(n=(16, 16, 16), amp=0.08, L=(1.0, 1.0, 1.0)):
    nx, ny, nz = n
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xs, ys, zs = I / nx, J / ny, K / nz
    s = np.sin(2 * math.pi * xs) * np.sin(2 * math.pi * ys) * np.sin(2 * math.pi * zs)
    xyz = np.stack([L[0] * (xs + amp * s), L[1] * (ys + amp * s), L[2] * (zs + amp * s)])
    per = [[L[0], 0, 0], [0, L[1], 0], [0, 0, L[2]]]
    return xyz, per


def uniform_flow_curvilinear(xyz, period, W0, gamma=1.4, bc=None):
    """Uniform primitive state W0 on a curvilinear grid (freestream preservation)."""
    nd = xyz.shape[0]
    shape = xyz.shape[1:]
    W = np.empty((nd + 2,) + shape)
    for v in range(nd + 2):
        W[v] = W0[v]
    n = list(shape[::-1])
    if bc is None:
        bc = [[PERIODIC, PERIODIC]] * nd
    return _problem("freestream", nd, n, [1.0] * nd, bc, W, gamma,
                    xyz=np.ascontiguousarray(xyz), period=period)


def field_on_curvilinear(xyz, period, W, gamma=1.4, bc=None):
    nd = xyz.shape[0]
    n = list(xyz.shape[1:][::-1])
    if bc is None:
        bc = [[PERIODIC, PERIODIC]] * nd
    return _problem("curvilinear", nd, n, [1.0] * nd, bc, W, gamma,
                    xyz=np.ascontiguousarray(xyz), period=period)


def batched_riemann(count=256, seed=0, n_lo=64, n_hi=512):
    """Batched 2D quadrant Riemann problems: sizes N ~ round(exp(U(ln n_lo, ln n_hi)))
    (square N x N), quadrant states as in random_quadrants, one seeded stream."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))).astype(int)
    return [random_quadrants(rng, int(n)) for n in sizes]
