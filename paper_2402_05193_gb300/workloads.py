"""Seeded synthetic workloads (initial conditions and case parameters).

Each generator returns a plain ``dict`` describing one simulation: grid,
boundary conditions, materials, scheme switches (``recon``, ``weno``,
``viscous``, ``limiter``; ``thinc`` and ``visc_order`` may be added), step
count, and the initial
PRIMITIVE field ``W`` of shape (nv, nz, ny, nx) in float64, with
nv = ndim + 2 (rho, u_d, p) for a single phase or ndim + 4
(a1*rho1, a2*rho2, u_d, p, a1) for the diffuse-interface model.  Primitive to
conservative conversion is left to whoever consumes the case (the GPU library
and the oracle each do their own), so this module holds no arithmetic of the
numerical method -- only the problem set-ups.

Cases follow the shapes of the paper's test problems (JAX-Fluids 2.0, arXiv
2402.05193): the two-Gaussian advection of §5.1, shock tubes of §5.3, the
helium shock-bubble set-up of §5.3.3, water shock-drop set-ups of §5.3.4, and
for the remaining benchmark configurations (Taylor-Green vortex,
Kelvin-Helmholtz layer) the standard textbook initial fields.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

PERIODIC, ZEROGRAD, SYMMETRY = "periodic", "zerograd", "symmetry"

# limiter tolerances of §3.3 (eps_rho, eps_rhoc2, eps_alpha)
EPS_FP64 = (1e-12, 1e-10, 1e-12)
EPS_FP32 = (1e-10, 1e-8, 1e-10)


def _case(name, *, ndim, n, dx, bc, W, model="spm", gamma=(1.4, 1.4), pinf=(0.0, 0.0),
          mu=0.0, Pr=0.72, R=1.0, recon="comp", viscous=False, limiter=False, cfl=0.5,
          fixed_dt=0.0, t_end=0.0, steps=1, lo=None, weno="js"):
    return dict(name=name, ndim=ndim, n=list(n), dx=list(dx), bc=[tuple(b) for b in bc],
                lo=list(lo) if lo is not None else [0.0] * ndim, model=model,
                gamma=tuple(gamma), pinf=tuple(pinf), mu=mu, Pr=Pr, R=R, recon=recon, weno=weno,
                viscous=viscous, limiter=limiter, cfl=cfl, fixed_dt=fixed_dt, t_end=t_end,
                steps=steps, W=np.ascontiguousarray(W, dtype=np.float64))


def _centres(n, lo, dx):
    return lo + (np.arange(n) + 0.5) * dx


def nvar(ndim: int, model: str) -> int:
    return ndim + (4 if model == "dim" else 2)


# ----------------------------------------------------------------- 1-D tubes --
def sod(n: int = 200):
    """Sod tube: x in [0,1], (rho,u,p) = (1,0,1) | (0.125,0,0.1) split at the
    face x = 0.5, gamma 1.4, zero-gradient ends, WENO5-JS (component) + HLLC +
    TVD-RK3, CFL 0.5, t_end 0.2."""
    dx = 1.0 / n
    x = _centres(n, 0.0, dx)
    W = np.zeros((3, 1, 1, n))
    left = x < 0.5
    W[0, 0, 0] = np.where(left, 1.0, 0.125)
    W[2, 0, 0] = np.where(left, 1.0, 0.1)
    return _case("sod", ndim=1, n=[n], dx=[dx], bc=[(ZEROGRAD, ZEROGRAD)], W=W, cfl=0.5,
                 t_end=0.2, steps=100000)


def two_material_tube(kind: str = "air_water", n: int = 200):
    """Two-fluid shock tubes of §5.3 with the diffuse-interface model (fluid 1
    on the left).  air_helium: x in [0,1], split 0.5, air (1,0,1, gamma 1.4)
    | helium (0.125,0,0.1, gamma 1.67), t = 0.15.  air_water: x in [0,1.5],
    split 0.8, water (1000,0,1e9, gamma 6.12, p_inf 3.43e8) | air
    (20,0,1e5, gamma 1.4); final time 1.5e-4 s (reading of the printed 0.15,
    taken in ms so that every wave stays inside the domain).  Volume fraction
    1-1e-8 / 1e-8 in the two phases."""
    if kind == "air_helium":
        L, x0, t_end = 1.0, 0.5, 0.15
        g, pi = (1.4, 1.67), (0.0, 0.0)
        left, right = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    elif kind == "air_water":
        L, x0, t_end = 1.5, 0.8, 1.5e-4
        g, pi = (6.12, 1.4), (3.43e8, 0.0)
        left, right = (1000.0, 0.0, 1e9), (20.0, 0.0, 1e5)
    else:
        raise ValueError(kind)
    dx = L / n
    x = _centres(n, 0.0, dx)
    a1 = np.where(x < x0, 1.0 - 1e-8, 1e-8)
    W = np.zeros((5, 1, 1, n))
    W[0, 0, 0] = a1 * left[0]
    W[1, 0, 0] = (1.0 - a1) * right[0]
    W[2, 0, 0] = np.where(x < x0, left[1], right[1])
    W[3, 0, 0] = np.where(x < x0, left[2], right[2])
    W[4, 0, 0] = a1
    c = _case(kind, ndim=1, n=[n], dx=[dx], bc=[(ZEROGRAD, ZEROGRAD)], W=W, model="dim",
              gamma=g, pinf=pi, recon="char", limiter=True, cfl=0.5, t_end=t_end,
              steps=100000)
    c["x0"] = x0
    c["states"] = (left, right)
    return c


def gaussians(n: int, t_end: float = 2.0, fixed_dt: float = 1e-5):
    """Advection of two Gaussians (§5.1): rho = 1 + 5 exp(-200 (x-0.5)^2) +
    5 exp(-200 (x-1.5)^2), u = 1, p = 1, gamma 1.4, x in [0,2] periodic; cell
    averages from the erf integral."""
    L = 2.0
    dx = L / n
    xf = np.arange(n + 1) * dx
    k = math.sqrt(200.0)

    def prim(xc):  # antiderivative of the two Gaussians
        return (5.0 * math.sqrt(math.pi) / (2.0 * k)) * (erf(k * (xc - 0.5)) + erf(k * (xc - 1.5)))

    rho = 1.0 + (prim(xf[1:]) - prim(xf[:-1])) / dx
    W = np.zeros((3, 1, 1, n))
    W[0, 0, 0] = rho
    W[1] = 1.0
    W[2] = 1.0
    return _case("gaussians", ndim=1, n=[n], dx=[dx], bc=[(PERIODIC, PERIODIC)], W=W,
                 fixed_dt=fixed_dt, t_end=t_end, steps=100000000)


# ------------------------------------------------------------------- 3-D TGV --
def tgv(n: int = 128, steps: int = 500):
    """Taylor-Green vortex on [0,2pi]^3, periodic, Ma 0.1, Re 1600, Pr 0.72,
    gamma 1.4: u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    p = p0 + (cos 2x + cos 2y)(cos 2z + 2)/16 with p0 = 1/(gamma Ma^2),
    isothermal rho = p/p0, mu = 1/1600, R = 1; WENO5-JS characteristic + HLLC
    + 4th-order viscous, CFL 0.5."""
    dx = 2.0 * math.pi / n
    x = _centres(n, 0.0, dx)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    gamma, Ma = 1.4, 0.1
    p0 = 1.0 / (gamma * Ma * Ma)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    W = np.empty((5, n, n, n))
    W[0] = p / p0
    W[1] = np.sin(X) * np.cos(Y) * np.cos(Z)
    W[2] = -np.cos(X) * np.sin(Y) * np.cos(Z)
    W[3] = 0.0
    W[4] = p
    return _case("tgv", ndim=3, n=[n] * 3, dx=[dx] * 3, bc=[(PERIODIC, PERIODIC)] * 3, W=W,
                 gamma=(gamma, gamma), mu=1.0 / 1600.0, Pr=0.72, R=1.0, recon="char",
                 viscous=True, cfl=0.5, steps=steps)


# ---------------------------------------------------------- 3-D shock bubble --
def shock_bubble(nx: int = 256, ny: int = 128, nz: int = 128, steps: int = 1000,
                 offset=(0.0, 0.0, 0.0)):
    """Air-helium shock-bubble interaction (diffuse interface; set-up after
    §5.3.3): dx = 1 mm, bubble radius 25 cells centred at cell (100, ny/2,
    nz/2) scaled with the grid, Ma 1.22 shock plane at x = 70 cells, post-shock
    air (1.6573, 114.5, 159056), pre-shock air (1.2041, 0, 101325), helium
    (0.1660, 0, 101325) with gamma 1.66; a_air = (1 + tanh((r-R)/dx))/2 clipped
    to [1e-8, 1-1e-8]; zero-gradient boundaries; limiters on; CFL 0.4.
    ``offset`` moves the bubble centre by that many cells (off the grid's
    mirror planes)."""
    s = nx / 256.0
    dx = 1e-3
    R = 25.0 * s * dx
    cx, cy, cz = ((100.0 * s + offset[0]) * dx, (0.5 * ny + offset[1]) * dx,
                  (0.5 * nz + offset[2]) * dx)
    xs = 70.0 * s * dx
    x = _centres(nx, 0.0, dx)
    y = _centres(ny, 0.0, dx)
    z = _centres(nz, 0.0, dx)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2)
    a_air = np.clip(0.5 * (1.0 + np.tanh((r - R) / dx)), 1e-8, 1.0 - 1e-8)
    post = X < xs
    rho_air = np.where(post, 1.6573, 1.2041)
    W = np.empty((7, nz, ny, nx))
    W[0] = a_air * rho_air
    W[1] = (1.0 - a_air) * 0.1660
    W[2] = np.where(post, 114.5, 0.0)
    W[3] = 0.0
    W[4] = 0.0
    W[5] = np.where(post, 159056.0, 101325.0)
    W[6] = a_air
    return _case("shock_bubble", ndim=3, n=[nx, ny, nz], dx=[dx] * 3,
                 bc=[(ZEROGRAD, ZEROGRAD)] * 3, W=W, model="dim", gamma=(1.4, 1.66),
                 pinf=(0.0, 0.0), recon="char", limiter=True, cfl=0.4, steps=steps)


# ------------------------------------------------------ 2-D batched drops -----
def _post_shock_air(Ma, rho1, p1, gamma=1.4):
    """Normal-shock (Rankine-Hugoniot) state behind a shock of Mach Ma moving
    into quiescent ideal gas (rho1, p1)."""
    m2 = Ma * Ma
    p2 = p1 * (1.0 + 2.0 * gamma / (gamma + 1.0) * (m2 - 1.0))
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    c1 = math.sqrt(gamma * p1 / rho1)
    u2 = Ma * c1 * (1.0 - rho1 / rho2)
    return rho2, u2, p2


def drop(N: int, radius: float, cx: float, cy: float, Ma: float):
    """One water drop (fluid 1: rho 1000, gamma 6.12, p_inf 3.43e8) in air
    (fluid 2: rho 1.2, gamma 1.4, p 1.01e5) on [0,1]^2 with N x N cells, hit by
    a Mach-Ma shock placed 0.05 left of the drop; tanh smear over 2 cells;
    zero-gradient boundaries; limiters on; CFL 0.4."""
    dx = 1.0 / N
    x = _centres(N, 0.0, dx)
    Y, X = np.meshgrid(x, x, indexing="ij")
    r = np.sqrt((X - cx) ** 2 + (Y - cy) ** 2)
    a1 = np.clip(0.5 * (1.0 - np.tanh((r - radius) / dx)), 1e-8, 1.0 - 1e-8)
    rho2, u2, p2 = _post_shock_air(Ma, 1.2, 1.01e5)
    post = X < cx - radius - 0.05
    W = np.empty((6, 1, N, N))
    W[0, 0] = a1 * 1000.0
    W[1, 0] = (1.0 - a1) * np.where(post, rho2, 1.2)
    W[2, 0] = np.where(post, u2, 0.0)
    W[3, 0] = 0.0
    W[4, 0] = np.where(post, p2, 1.01e5)
    W[5, 0] = a1
    return _case("drop", ndim=2, n=[N, N], dx=[dx, dx], bc=[(ZEROGRAD, ZEROGRAD)] * 2, W=W,
                 model="dim", gamma=(6.12, 1.4), pinf=(3.43e8, 0.0), recon="char",
                 limiter=True, cfl=0.4, steps=200)


def drop_batch(nsim: int = 96, seed: int = 1234, sizes=(64, 128, 192, 256)):
    """nsim independent drops of uneven sizes: N uniform from ``sizes``, radius
    ~ U(0.08, 0.15), centre x ~ U(0.4, 0.6), y ~ U(0.35, 0.65), shock Mach
    ~ U(1.2, 2.4); numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(nsim):
        N = int(rng.choice(sizes))
        radius = rng.uniform(0.08, 0.15)
        cx = rng.uniform(0.4, 0.6)
        cy = rng.uniform(0.35, 0.65)
        Ma = rng.uniform(1.2, 2.4)
        cases.append(drop(N, radius, cx, cy, Ma))
    return cases


# --------------------------------------------------------------- 2-D KH -------
def kelvin_helmholtz(n: int = 256, seed: int = 7, steps: int = 2000):
    """Periodic double shear layer on [0,1]^2: rho = 1 + (tanh((y-1/4)/0.01)
    - tanh((y-3/4)/0.01))/2, u = -1/2 + (same bracket)/2, p = 2.5, v = 0.01
    * (1/4) sum_{k=1..4} sin(2 pi k x + phi_k) (g(y-1/4) + g(y-3/4)) with
    g(s) = exp(-s^2/(2*0.05^2)), phi_k ~ U(0, 2pi) from default_rng(seed);
    gamma 1.4, inviscid WENO5-JS + HLLC."""
    rng = np.random.default_rng(seed)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=4)
    dx = 1.0 / n
    x = _centres(n, 0.0, dx)
    Y, X = np.meshgrid(x, x, indexing="ij")
    br = np.tanh((Y - 0.25) / 0.01) - np.tanh((Y - 0.75) / 0.01)
    g = np.exp(-((Y - 0.25) ** 2) / (2 * 0.05 ** 2)) + np.exp(-((Y - 0.75) ** 2) / (2 * 0.05 ** 2))
    v = np.zeros_like(X)
    for k in range(4):
        v += np.sin(2.0 * math.pi * (k + 1) * X + phi[k])
    v *= 0.01 * 0.25 * g
    W = np.empty((4, 1, n, n))
    W[0, 0] = 1.0 + 0.5 * br
    W[1, 0] = -0.5 + 0.5 * br
    W[2, 0] = v
    W[3, 0] = 2.5
    return _case("kelvin_helmholtz", ndim=2, n=[n, n], dx=[dx, dx],
                 bc=[(PERIODIC, PERIODIC)] * 2, W=W, recon="comp", cfl=0.5, steps=steps)


# ------------------------------------------------------ generic random fields --
def smooth_random(ndim: int, n, model: str = "spm", seed: int = 0, bc=PERIODIC,
                  amp: float = 0.1, recon: str = "char", viscous: bool = False,
                  limiter: bool = False, pinf=(0.0, 0.0), gamma=(1.4, 1.4), mu: float = 0.0,
                  rho=(1.0, 0.5), p0: float = 1.0, u0: float = 0.3):
    """Smooth random periodic perturbation of a uniform state (Fourier modes
    1..3 with seeded amplitudes and phases) on the unit box; for the diffuse
    interface model a smooth volume-fraction blob between the two fluids.
    ``rho`` = reference densities of fluids 1 and 2, ``p0`` the reference
    pressure, ``u0`` the mean velocity (perturbations scale with them)."""
    rng = np.random.default_rng(seed)
    n = list(n)
    dx = [1.0 / m for m in n]
    axes = [_centres(n[e], 0.0, dx[e]) for e in range(ndim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]  # grids[e] varies along axis e
    shp = tuple([n[e] for e in range(ndim)][::-1])
    shp4 = (1,) * (3 - ndim) + shp

    def field():
        f = np.zeros(shp)
        for _ in range(3):
            k = rng.integers(1, 4, size=ndim)
            ph = rng.uniform(0, 2 * math.pi)
            arg = sum(2 * math.pi * k[e] * grids[e] for e in range(ndim))
            f += rng.uniform(-1, 1) * np.sin(arg + ph)
        return f.reshape(shp4) / 3.0

    nv = nvar(ndim, model)
    W = np.empty((nv,) + shp4)
    if model == "spm":
        W[0] = rho[0] * (1.0 + amp * field())
        for d in range(ndim):
            W[1 + d] = u0 * (1.0 + 5.0 * amp * field())
        W[1 + ndim] = p0 * (1.0 + amp * field())
    else:
        a1 = np.clip(0.5 + 0.45 * field() * 3.0 / 2.0, 1e-8, 1.0 - 1e-8)
        W[0] = a1 * rho[0] * (1.0 + amp * field())
        W[1] = (1.0 - a1) * rho[1] * (1.0 + amp * field())
        for d in range(ndim):
            W[2 + d] = u0 * (1.0 + 5.0 * amp * field())
        W[2 + ndim] = p0 * (1.0 + amp * field())
        W[3 + ndim] = a1
    return _case("smooth_random", ndim=ndim, n=n, dx=dx, bc=[(bc, bc)] * ndim, W=W, model=model,
                 gamma=gamma, pinf=pinf, mu=mu, recon=recon, viscous=viscous, limiter=limiter,
                 cfl=0.5, steps=1)


# ------------------------------------------------------ level-set transport --
def levelset_sphere(n: int = 128):
    """Level-set transport workload: the signed distance phi = R - |x - c| of
    a sphere of radius 1/4 centred at (0.5, 0.6, 0.5) in the unit cube (n^3
    cubic cells, zero-gradient sides), carried by the solid-body rotation
    u = (-(y - 0.5), x - 0.5, 0) about the cube's z axis; dt = 0.5 h /
    max|u|.  Returns a dict with phi (n, n, n), vel (3, n, n, n), h, dt and
    the boundary conditions."""
    h = 1.0 / n
    x = _centres(n, 0.0, h)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi = 0.25 - np.sqrt((X - 0.5) ** 2 + (Y - 0.6) ** 2 + (Z - 0.5) ** 2)
    vel = np.stack([-(Y - 0.5), X - 0.5, np.zeros_like(X)])
    umax = float(np.sqrt(vel[0] ** 2 + vel[1] ** 2).max())
    return {"name": "levelset_sphere", "n": [n, n, n], "h": h, "phi": phi, "vel": vel,
            "dt": 0.5 * h / umax, "bc": [(ZEROGRAD, ZEROGRAD)] * 3}


def levelset_drop(n: int = 128) -> dict:
    """Two-phase level-set workload on n^3 periodic cubic cells (unit box):
    a drop of a stiffened gas (gamma 4.4, p_inf 6, density 5; phase 1,
    phi > 0) of radius 1/4 in an ideal gas (gamma 1.4, density 1; phase 2),
    both moving with u = (0.4, 0.3, 0.2) at pressure 1; dt at CFL 0.3 of
    the faster phase's |u| + c.  Returns phi (n, n, n), W1, W2 (5, n, n, n:
    rho, u, v, w, p in every cell), the materials, h, dt and bc."""
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi = 0.25 - np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    u = (0.4, 0.3, 0.2)
    one = np.ones_like(phi)
    W1 = np.stack([5.0 * one] + [c * one for c in u] + [one])
    W2 = np.stack([one] + [c * one for c in u] + [one])
    mat1, mat2 = (4.4, 6.0), (1.4, 0.0)
    umag = float(np.sqrt(sum(c * c for c in u)))
    smax = umag + max(np.sqrt(4.4 * (1.0 + 6.0) / 5.0), np.sqrt(1.4))
    return {"phi": phi, "W1": W1, "W2": W2, "mat1": mat1, "mat2": mat2, "h": h, "dt": 0.3 * h / smax,
            "n": [n, n, n], "bc": [("periodic", "periodic")] * 3}
