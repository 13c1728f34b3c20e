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


# ---------------------------------------------------------------- viscous cases
PRANDTL = 0.72


def _viscous(d, re, minf, suth=0.0, twall=1.0, pr=PRANDTL):
    d.update(viscous=1, re=float(re), minf=float(minf), suth=float(suth), twall=float(twall), pr=float(pr))
    return d


def shear_wave(n=32, amp=1e-3, minf=0.2, re=100.0, suth=0.0):
    """2D periodic shear wave u = amp sin(2 pi y), v = 0, rho = 1, p = 1/(gamma M^2)
    (T = 1) on [0,1]^2: a linear viscous decay at rate nu (2 pi)^2."""
    gamma = 1.4
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    W = np.zeros((4, n, n))
    W[0] = 1.0
    W[1] = amp * np.sin(2 * math.pi * Y)
    W[3] = 1.0 / (gamma * minf * minf)
    d = _problem("shear_wave", 2, [n, n], [h, h], [[PERIODIC, PERIODIC]] * 2, W, gamma, amp=amp)
    return _viscous(d, re, minf, suth)


def wall_channel(n=32, nx=8, minf=0.5, re=50.0, suth=0.5, twall=1.0, fields=None, bc_y=None):
    """2D channel [0, nx/n] x [0,1] (x periodic) with isothermal no-slip walls at
    y = 0 and y = 1 (bc_y overrides).  fields(X, Y) -> (u, v, p, T) primitive
    profiles; default: u = 1e-3 sin(pi y), v = 0, p = 1/(gamma M^2), T = twall."""
    gamma = 1.4
    h = 1.0 / n
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, y)
    if fields is None:
        u, v = 1e-3 * np.sin(math.pi * Y), 0.0 * Y
        p, T = np.full_like(Y, 1.0 / (gamma * minf * minf)), np.full_like(Y, twall)
    else:
        u, v, p, T = fields(X, Y)
    W = np.stack([gamma * minf * minf * p / T, u, v, p])
    bc = [[PERIODIC, PERIODIC], bc_y if bc_y is not None else [WALL, WALL]]
    d = _problem("wall_channel", 2, [nx, n], [h, h], bc, W, gamma)
    return _viscous(d, re, minf, suth, twall)


WALL = 4


def compression_ramp(nx=768, ny=192, nz=128, mach=2.9, re_theta=2400.0, angle_deg=24.0, corner=0.4,
                     Lx=534.6, Ly=161.0, Lz=61.2, delta=20.4, cf=2.2e-3, t_inf_kelvin=108.1,
                     noise=0.05, seed=0, cfl=0.2):
    """3D supersonic compression ramp (Sec. 3.3, M = 2.9, 24 degrees), lengths in
    units of the inflow momentum thickness theta (so Re = Re_theta):

    * body-fitted algebraic grid, uniform in x and z.  The wall y_w(x) is flat
      up to x_c = corner * Lx, then rises at the ramp angle (corner rounded
      over four cells).  Wall-normal lines are vertical; node rows sit at
      eta_j = (j + 1/2) / ny of the tanh stretching
      y = y_w + Ly (1 + tanh(b (eta - 1)) / tanh(b)), with b chosen so that the
      first row is at half the viscous length nu_w / u_tau above the wall
      (a first cell of y+ = 1, the wall face half-way between row 0 and its
      mirror ghost).  u_tau comes from an assumed skin friction cf with the
      wall density and Sutherland viscosity;
    * wall temperature 1.14 times the recovery temperature (recovery factor
      0.89), Sutherland constant 110.4 K / T_inf, Pr = 0.72;
    * mean boundary layer of thickness delta: u = min((y_n/delta)^{1/7},
      y_n u_tau^2 / nu_w) (power law over a linear sublayer), Crocco-Busemann
      temperature, uniform pressure, flow along the local wall direction, with
      y_n = y - y_w(x); the initial state is this mean flow;
    * inflow plane (x = 0): the mean profile plus seeded uniform velocity
      fluctuations of amplitude noise * 4 u (1 - u) (frozen in time);
    * boundaries: x inflow profile / supersonic outflow (extrapolation),
      y isothermal wall / extrapolation, z periodic."""
    gamma = 1.4
    suth = 110.4 / t_inf_kelvin
    t_rec = 1.0 + 0.89 * 0.5 * (gamma - 1.0) * mach * mach
    t_wall = 1.14 * t_rec
    mu_w = t_wall ** 1.5 * (1.0 + suth) / (t_wall + suth)
    rho_w = 1.0 / t_wall
    u_tau = math.sqrt(0.5 * cf / rho_w)
    nu_w = mu_w / (re_theta * rho_w)
    dy1 = nu_w / u_tau
    eta = (np.arange(ny) + 0.5) / ny

    def row0(b):
        return Ly * (1.0 + math.tanh(b * (eta[0] - 1.0)) / math.tanh(b))

    lo, hi = 1e-3, 30.0
    for _ in range(200):  # bisection: row0 decreases as b grows
        mid = 0.5 * (lo + hi)
        if row0(mid) > 0.5 * dy1:
            lo = mid
        else:
            hi = mid
    b = 0.5 * (lo + hi)
    s = 1.0 + np.tanh(b * (eta - 1.0)) / math.tanh(b)
    x = np.arange(nx) * (Lx / (nx - 1.0))
    z = np.arange(nz) * (Lz / nz)
    xc = corner * Lx
    w = 4.0 * Lx / (nx - 1.0)
    ta = math.tan(math.radians(angle_deg))
    yw = ta * w * np.logaddexp(0.0, (x - xc) / w)
    yw = yw - yw[0]
    Z, S, X = np.meshgrid(z, s, x, indexing="ij")
    YW = np.broadcast_to(yw[None, None, :], X.shape)
    Y = YW + Ly * S
    xyz = np.stack([X, Y, Z])
    yn = Y - YW
    ubl = np.minimum(np.clip(yn / delta, 0.0, 1.0) ** (1.0 / 7.0), yn * u_tau * u_tau / nu_w)
    T = t_wall + (t_rec - t_wall) * ubl + (1.0 - t_rec) * ubl * ubl
    p0 = 1.0 / (gamma * mach * mach)
    slope = np.gradient(yw, x)
    cth = 1.0 / np.sqrt(1.0 + slope * slope)
    sth = slope * cth
    u = ubl * cth[None, None, :]
    v = ubl * sth[None, None, :]
    p = np.full_like(T, p0)
    W = np.stack([gamma * mach * mach * p / T, u, v, np.zeros_like(u), p])
    # inflow plane: mean profile at x = 0 plus frozen seeded fluctuations
    rng = np.random.default_rng(seed)
    Win = W[:, :, :, 0].copy()
    amp = noise * 4.0 * ubl[:, :, 0] * (1.0 - ubl[:, :, 0])
    Win[1:4] += rng.uniform(-1.0, 1.0, size=(3,) + amp.shape) * amp
    n = [nx, ny, nz]
    period = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, Lz]]
    d = _problem("compression_ramp", 3, n, [1.0, 1.0, 1.0],
                 [[INFLOW, EXTRAP], [WALL, EXTRAP], [PERIODIC, PERIODIC]], W, gamma,
                 xyz=np.ascontiguousarray(xyz), period=period, cfl=cfl, t_wall=t_wall, dy1=dy1,
                 stretch=b, suth_kelvin=110.4, t_inf_kelvin=t_inf_kelvin)
    d["inflow_profile"] = {(0, 0): np.ascontiguousarray(Win.reshape(5, -1))}
    d["inflow"] = {(0, 0): (1.0, 1.0, 0.0, 0.0, p0)}
    return _viscous(d, re_theta, mach, suth, t_wall)
