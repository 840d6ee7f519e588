"""CPU oracle of the JAX-Fluids 2.0 finite-volume scheme (test infrastructure).

A plain, slow FP64 C++ implementation of what the GPU library computes, built
from the paper (arXiv 2402.05193) alone and sharing no code with the CUDA
path.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  prim/cons conversion, mixture EOS   closed forms, pure-phase reduction
  WENO5-JS                            polynomial exactness, linear weights
  characteristic projection           K K^-1 = I, component equivalence
  HLLC                                consistency, upwinding, symmetry,
                                      stationary contact
  rhs / rk3 / run                     exact Riemann solution (Sod),
                                      5th-order convergence, conservation,
                                      mirror symmetry, uniform-flow invariance
  viscous flux                        manufactured linear / cubic fields
  cfl dt                              closed form on a uniform state
  interpolation / flux limiter        single-face decisions worked out by
                                      hand (each check, its tolerance, the
                                      test states U_i -/+ lam F with
                                      lam = 2 D dt/dx_d, the volume
                                      fraction's source share); both fire
                                      in the two-material tubes
  tangent (dual numbers)              central finite differences
  exact Riemann solver                Rankine-Hugoniot and isentropic
                                      relations, textbook Sod star state
  level set: apertures, volume        exact areas / volumes of planar
  fraction, interface segment,        interfaces, second-order sphere and
  normal (App. D)                     circle convergence, plane normals
  level-set advection (§3.5)          degree-5 exactness, fifth-order
                                      convergence of a carried profile
  reinitialisation (§3.5)             WENO-HJ3 exact for quadratics and
                                      third order; a plane's distance is a
                                      fixed point; twice a distance regains
                                      |grad phi| = 1 near the interface
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_SOURCES = ["orc.cpp", "orc_riemann.cpp", "orc_levelset.cpp"]
_HEADERS = ["orc.h", "orc_scheme.hpp", "orc_types.hpp"]
_lock = threading.Lock()

SPM, DIM = 0, 1
COMP, CHAR = 0, 1
PERIODIC, ZEROGRAD, SYMMETRY = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, no fast-math)."""
    with _lock:
        srcs = [os.path.join(_HERE, s) for s in _SOURCES]
        deps = srcs + [os.path.join(_HERE, h) for h in _HEADERS]
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= max(os.path.getmtime(p) for p in deps)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", tmp] + srcs
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class Config(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("dx", ctypes.c_double * 3),
        ("bc", (ctypes.c_int * 2) * 3),
        ("model", ctypes.c_int),
        ("gamma", ctypes.c_double * 2),
        ("pinf", ctypes.c_double * 2),
        ("mu", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("R", ctypes.c_double),
        ("recon", ctypes.c_int),
        ("viscous", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("cfl", ctypes.c_double),
        ("fixed_dt", ctypes.c_double),
        ("t_end", ctypes.c_double),
        ("eps_rho", ctypes.c_double),
        ("eps_rhoc2", ctypes.c_double),
        ("eps_alpha", ctypes.c_double),
        ("weno_eps", ctypes.c_double),
        ("weno_z", ctypes.c_int),
        ("thinc", ctypes.c_int),
        ("visc_order", ctypes.c_int),
        ("teno", ctypes.c_int),
    ]


class Counts(ctypes.Structure):
    _fields_ = [("il_sides", ctypes.c_longlong), ("fl_faces", ctypes.c_longlong)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        cp = ctypes.POINTER(Config)
        L.orc_nvar.argtypes = [cp]
        L.orc_prim_to_cons.argtypes = [cp, dp, dp]
        L.orc_cons_to_prim.argtypes = [cp, dp, dp]
        L.orc_rhs.argtypes = [cp, dp, ctypes.c_double, dp, ctypes.POINTER(Counts)]
        L.orc_dt.argtypes = [cp, dp, ctypes.c_double]
        L.orc_dt.restype = ctypes.c_double
        L.orc_rk3.argtypes = [cp, dp, ctypes.c_double, ctypes.POINTER(Counts)]
        L.orc_run.argtypes = [cp, dp, ctypes.c_int, dp, dp, ctypes.POINTER(Counts)]
        L.orc_run.restype = ctypes.c_int
        L.orc_sums.argtypes = [cp, dp, dp]
        L.orc_rhs_tangent.argtypes = [cp, dp, dp, ctypes.c_double, dp, dp]
        L.orc_run_tangent.argtypes = [cp, dp, dp, ctypes.c_int, ctypes.c_double]
        L.orc_count_flops.argtypes = [cp, dp, ctypes.c_double, dp]
        L.orc_exact_riemann.argtypes = [ctypes.c_double] * 10 + [
            dp, ctypes.c_int, dp, dp, dp, ctypes.POINTER(ctypes.c_int), dp]
        L.orc_exact_riemann.restype = ctypes.c_int
        L.orc_weno5js.argtypes = [dp, ctypes.c_double]
        L.orc_weno5js.restype = ctypes.c_double
        L.orc_weno5z.argtypes = [dp, ctypes.c_double]
        L.orc_weno5z.restype = ctypes.c_double
        L.orc_weno5_weights.argtypes = [dp, ctypes.c_double, ctypes.c_int, dp]
        L.orc_teno6a.argtypes = [dp, dp]
        L.orc_teno6a.restype = ctypes.c_double
        d_ = ctypes.c_double
        L.orc_thinc_fit.argtypes = [d_, d_, d_, d_, dp, dp, dp]
        L.orc_thinc_fit.restype = ctypes.c_int
        L.orc_thinc_face.argtypes = [d_, d_, d_, d_, ctypes.c_int, dp]
        L.orc_thinc_face.restype = ctypes.c_int
        L.orc_thinc_normals.argtypes = [cp, dp, dp]
        L.orc_reconstruct.argtypes = [cp, ctypes.c_int, dp, dp, dp]
        L.orc_hllc.argtypes = [cp, ctypes.c_int, dp, dp, dp, dp]
        L.orc_interp_limit.argtypes = [cp, dp, dp]
        L.orc_interp_limit.restype = ctypes.c_int
        L.orc_flux_limit_test.argtypes = [cp, ctypes.c_int, ctypes.c_double, dp, ctypes.c_double, dp, dp]
        L.orc_flux_limit_test.restype = ctypes.c_int
        L.orc_ls_nface.argtypes = [cp]
        L.orc_ls_nface.restype = ctypes.c_longlong
        L.orc_ls_geometry.argtypes = [cp, dp, dp, dp, dp, dp]
        L.orc_ls_geometry.restype = ctypes.c_int
        L.orc_ls_face_fraction.argtypes = [dp]
        L.orc_ls_face_fraction.restype = ctypes.c_double
        L.orc_ls_rhs.argtypes = [cp, dp, dp, dp]
        L.orc_ls_rhs.restype = ctypes.c_int
        L.orc_ls_advect.argtypes = [cp, dp, dp, ctypes.c_double, ctypes.c_int]
        L.orc_ls_advect.restype = ctypes.c_int
        L.orc_ls_reinit_rhs.argtypes = [cp, dp, dp, ctypes.c_double, dp]
        L.orc_ls_reinit_rhs.restype = ctypes.c_int
        L.orc_ls_reinit.argtypes = [cp, dp, ctypes.c_int, ctypes.c_double]
        L.orc_ls_reinit.restype = ctypes.c_int
        L.orc_ls_weno3_hj.argtypes = [dp, ctypes.c_double, dp, dp]
        L.orc_ls_count_flops.argtypes = [cp, dp, dp, dp]
        L.orc_ls_count_flops.restype = ctypes.c_int
        L.orc_ls_interface_riemann.argtypes = [dp, dp, dp]
        L.orc_ls_interface_quantities.argtypes = [cp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_ls_interface_quantities.restype = ctypes.c_int
        L.orc_ls_extend.argtypes = [cp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.orc_ls_extend.restype = ctypes.c_int
        L.orc_ls_cut_rhs.argtypes = [cp, dp, dp, ctypes.c_int, dp, dp, dp]
        L.orc_ls_cut_rhs.restype = ctypes.c_int
        L.orc_ls_mix.argtypes = [cp, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp]
        L.orc_ls_mix.restype = ctypes.c_int
        L.orc_ls_init.argtypes = [cp, cp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_ls_init.restype = ctypes.c_int
        L.orc_ls_step.argtypes = [cp, cp, ctypes.c_double, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp, dp, dp]
        L.orc_ls_step.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_config(*, ndim, n, dx, bc, model=SPM, gamma=(1.4, 1.4), pinf=(0.0, 0.0),
                mu=0.0, Pr=0.72, R=1.0, recon=COMP, viscous=False, limiter=False,
                cfl=0.5, fixed_dt=0.0, t_end=0.0, eps=None, weno_eps=1e-6,
                weno="js", thinc=False, visc_order=4) -> Config:
    """Build an oracle configuration.  ``eps`` = (eps_rho, eps_rhoc2, eps_alpha);
    the default is the paper's double-precision set (§3.3).  ``weno`` = "js"
    (Jiang-Shu weights), "z" (Borges et al. WENO5-Z weights) or "teno6a"
    (the TENO6-A reconstruction of the paper's single-phase runs); ``thinc``
    turns on the THINC reconstruction of the volume fraction (five-equation
    model); ``visc_order`` (2, 4, 6) is the order of the central dissipative
    stencils."""
    if visc_order not in (2, 4, 6):
        raise ValueError("visc_order must be 2, 4 or 6")
    if weno not in ("js", "z", "teno6a"):
        raise ValueError("weno must be 'js', 'z' or 'teno6a'")
    c = Config()
    c.ndim = ndim
    nn = list(n) + [1] * (3 - len(n))
    dd = list(dx) + [1.0] * (3 - len(dx))
    for e in range(3):
        c.n[e] = nn[e]
        c.dx[e] = dd[e]
        b = bc[e] if e < len(bc) else (ZEROGRAD, ZEROGRAD)
        c.bc[e][0], c.bc[e][1] = b
    c.model = model
    c.gamma[0], c.gamma[1] = gamma
    c.pinf[0], c.pinf[1] = pinf
    c.mu, c.Pr, c.R = mu, Pr, R
    c.recon = recon
    c.viscous = int(viscous)
    c.limiter = int(limiter)
    c.cfl, c.fixed_dt, c.t_end = cfl, fixed_dt, t_end
    e = eps if eps is not None else (1e-12, 1e-10, 1e-12)
    c.eps_rho, c.eps_rhoc2, c.eps_alpha = e
    c.weno_eps = weno_eps
    c.weno_z = 1 if weno == "z" else 0
    c.teno = 1 if weno == "teno6a" else 0
    c.thinc = 1 if thinc else 0
    c.visc_order = visc_order
    return c


def nvar(c: Config) -> int:
    return lib().orc_nvar(ctypes.byref(c))


def shape(c: Config):
    """(nv, nz, ny, nx) of a state array."""
    n = [c.n[e] if e < c.ndim else 1 for e in range(3)]
    return (nvar(c), n[2], n[1], n[0])


def prim_to_cons(c: Config, W: np.ndarray) -> np.ndarray:
    W = np.ascontiguousarray(W, dtype=np.float64)
    U = np.empty_like(W)
    lib().orc_prim_to_cons(ctypes.byref(c), _p(W), _p(U))
    return U


def cons_to_prim(c: Config, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    W = np.empty_like(U)
    lib().orc_cons_to_prim(ctypes.byref(c), _p(U), _p(W))
    return W


def rhs(c: Config, U: np.ndarray, dt: float = 0.0):
    """R(U) and the limiter counters."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    R = np.empty_like(U)
    cnt = Counts()
    lib().orc_rhs(ctypes.byref(c), _p(U), dt, _p(R), ctypes.byref(cnt))
    return R, (cnt.il_sides, cnt.fl_faces)


def dt(c: Config, U: np.ndarray, t: float = 0.0) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64)
    return lib().orc_dt(ctypes.byref(c), _p(U), t)


def rk3(c: Config, U: np.ndarray, dt_: float):
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    cnt = Counts()
    lib().orc_rk3(ctypes.byref(c), _p(U), dt_, ctypes.byref(cnt))
    return U, (cnt.il_sides, cnt.fl_faces)


def run(c: Config, U: np.ndarray, nsteps: int, t: float = 0.0):
    """nsteps CFL (or fixed-dt) RK3 steps.  Returns (U, t, steps taken,
    last dt, (il_sides, fl_faces))."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    tt = ctypes.c_double(t)
    dl = ctypes.c_double(0.0)
    cnt = Counts()
    k = lib().orc_run(ctypes.byref(c), _p(U), nsteps, ctypes.byref(tt), ctypes.byref(dl),
                      ctypes.byref(cnt))
    return U, tt.value, k, dl.value, (cnt.il_sides, cnt.fl_faces)


def sums(c: Config, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.empty(nvar(c))
    lib().orc_sums(ctypes.byref(c), _p(U), _p(out))
    return out


def rhs_tangent(c: Config, U: np.ndarray, Ud: np.ndarray, dt_: float = 0.0):
    U = np.ascontiguousarray(U, dtype=np.float64)
    Ud = np.ascontiguousarray(Ud, dtype=np.float64)
    R = np.empty_like(U)
    Rd = np.empty_like(U)
    lib().orc_rhs_tangent(ctypes.byref(c), _p(U), _p(Ud), dt_, _p(R), _p(Rd))
    return R, Rd


def run_tangent(c: Config, U: np.ndarray, Ud: np.ndarray, nsteps: int, dt_: float):
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    Ud = np.array(Ud, dtype=np.float64, order="C", copy=True)
    lib().orc_run_tangent(ctypes.byref(c), _p(U), _p(Ud), nsteps, dt_)
    return U, Ud


def count_flops(c: Config, U: np.ndarray, dt_: float = 0.0) -> dict:
    """Algorithmic flops per interior cell (see orc.h for the categories)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    out = np.zeros(10)
    lib().orc_count_flops(ctypes.byref(c), _p(U), dt_, _p(out))
    ncell = int(np.prod(shape(c)[1:]))
    keys = ["face_x", "face_y", "face_z", "divergence", "cons2prim", "rk_stage", "cfl",
            "div_count", "sqrt_count", "interface_normal"]
    return {k: out[i] / ncell for i, k in enumerate(keys)}


def weno5js(v, eps: float = 1e-6) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.size == 5
    return lib().orc_weno5js(_p(v), eps)


def weno5z(v, eps: float = 1e-6) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.size == 5
    return lib().orc_weno5z(_p(v), eps)


def teno6a(v) -> float:
    """TENO6-A value at x_{i+1/2} from the left for v = v_{i-2..i+3}."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.size == 6
    return lib().orc_teno6a(_p(v), None)


def teno6a_parts(v) -> dict:
    """The steps of teno6a: candidates q, smoothness indicators beta (and
    beta6 of all six cells), scale-separation weights chi, stencil flags
    delta and the cut-off C_T."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.size == 6
    out = np.zeros(18)
    val = lib().orc_teno6a(_p(v), _p(out))
    return {"value": val, "q": out[0:4].copy(), "beta": out[4:8].copy(), "chi": out[8:12].copy(),
            "delta": out[12:16].astype(int), "ct": out[16], "beta6": out[17]}


def weno5_weights(v, eps: float = 1e-6, weno: str = "js") -> np.ndarray:
    """Normalised nonlinear weights (omega_0, omega_1, omega_2) of the value
    from the left for v = v_{i-2..i+2}."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert v.size == 5
    out = np.zeros(3)
    lib().orc_weno5_weights(_p(v), eps, 1 if weno == "z" else 0, _p(out))
    return out


def thinc_fit(am: float, ac: float, ap: float, nabs: float):
    """(theta, beta, xc) of the THINC profile of an interface cell, else None."""
    th, be, xc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    ok = lib().orc_thinc_fit(am, ac, ap, nabs, ctypes.byref(th), ctypes.byref(be), ctypes.byref(xc))
    return (th.value, be.value, xc.value) if ok else None


def thinc_face(am: float, ac: float, ap: float, nabs: float, side: int):
    """THINC face value of an interface cell (side 0: xi = 1, side 1: xi = 0),
    else None."""
    out = ctypes.c_double()
    ok = lib().orc_thinc_face(am, ac, ap, nabs, side, ctypes.byref(out))
    return out.value if ok else None


def thinc_normals(c: Config, W: np.ndarray) -> np.ndarray:
    """|n_d| of every cell, shape (ndim, nz, ny, nx)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    sh = shape(c)
    out = np.zeros((c.ndim,) + tuple(sh[1:]))
    lib().orc_thinc_normals(ctypes.byref(c), _p(W), _p(out))
    return out


def reconstruct(c: Config, d: int, Ws: np.ndarray):
    """Left/right primitive face states of axis d from the (6, nv) stencil."""
    Ws = np.ascontiguousarray(Ws, dtype=np.float64)
    nv = nvar(c)
    assert Ws.shape == (6, nv)
    WL, WR = np.empty(nv), np.empty(nv)
    lib().orc_reconstruct(ctypes.byref(c), d, _p(Ws), _p(WL), _p(WR))
    return WL, WR


def hllc(c: Config, d: int, WL, WR):
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    F = np.empty(nvar(c))
    uh = ctypes.c_double(0.0)
    lib().orc_hllc(ctypes.byref(c), d, _p(WL), _p(WR), _p(F),
                   ctypes.cast(ctypes.pointer(uh), ctypes.POINTER(ctypes.c_double)))
    return F, uh.value


def interp_limit(c: Config, Wf, W1):
    """Interpolation limiter of one face side: (switched, the side's state
    after the limiter), from the reconstructed primitive state Wf and the
    first-order cell state W1."""
    Wf = np.array(Wf, dtype=np.float64, copy=True)
    W1 = np.ascontiguousarray(W1, dtype=np.float64)
    assert Wf.shape == W1.shape == (nvar(c),)
    k = lib().orc_interp_limit(ctypes.byref(c), _p(Wf), _p(W1))
    return bool(k), Wf


def flux_limit_test(c: Config, d: int, dt_: float, F, uh: float, Ui, Uj) -> bool:
    """Flux-limiter test of a face of axis d: True if the face flux F (with
    upwinded velocity uh) makes a test state of the conservative cell states
    Ui, Uj inadmissible over the step dt."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    Ui = np.ascontiguousarray(Ui, dtype=np.float64)
    Uj = np.ascontiguousarray(Uj, dtype=np.float64)
    assert F.shape == Ui.shape == Uj.shape == (nvar(c),)
    return bool(lib().orc_flux_limit_test(ctypes.byref(c), d, float(dt_), _p(F), float(uh), _p(Ui), _p(Uj)))


def exact_riemann(left, right, xi):
    """left/right = (gamma, pinf, rho, u, p).  Returns rho, u, p, material
    (0 left / 1 right) at xi = (x - x0)/t, and (p*, u*, rho*_L, rho*_R)."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    n = xi.size
    rho, u, p = np.empty(n), np.empty(n), np.empty(n)
    mat = np.empty(n, dtype=np.int32)
    star = np.empty(4)
    it = lib().orc_exact_riemann(*[float(v) for v in left], *[float(v) for v in right],
                                 _p(xi), n, _p(rho), _p(u), _p(p),
                                 mat.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(star))
    if it < 0:
        raise RuntimeError("exact Riemann iteration failed")
    return rho, u, p, mat, tuple(star)


# ---------------------------------------------------------------- level set --
def ls_config(*, ndim, n, h, bc):
    """Grid of cubic cells (size h) for the level-set functions."""
    return make_config(ndim=ndim, n=n, dx=[h] * ndim, bc=bc)


def _ls_check(r: int):
    if r != 0:
        raise ValueError("level-set oracle: the grid must be 2-D or 3-D with cubic cells")


def ls_nface(c: Config) -> int:
    return int(lib().orc_ls_nface(ctypes.byref(c)))


def ls_geometry(c: Config, phi: np.ndarray):
    """Apertures (concatenated face arrays of every axis), volume fraction,
    interface segment and normal (ndim cell arrays) of the positive phase."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    nc = phi.size
    ap = np.zeros(max(ls_nface(c), 0))
    alpha, dg = np.zeros(nc), np.zeros(nc)
    nrm = np.zeros(c.ndim * nc)
    _ls_check(lib().orc_ls_geometry(ctypes.byref(c), _p(phi), _p(ap), _p(alpha), _p(dg), _p(nrm)))
    return ap, alpha.reshape(phi.shape), dg.reshape(phi.shape), nrm.reshape((c.ndim,) + phi.shape)


def ls_face_fraction(p4) -> float:
    p = np.ascontiguousarray(p4, dtype=np.float64)
    return float(lib().orc_ls_face_fraction(_p(p)))


def ls_rhs(c: Config, phi: np.ndarray, vel: np.ndarray) -> np.ndarray:
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    out = np.zeros_like(phi)
    _ls_check(lib().orc_ls_rhs(ctypes.byref(c), _p(phi), _p(vel), _p(out)))
    return out


def ls_advect(c: Config, phi: np.ndarray, vel: np.ndarray, dt_: float, nsteps: int) -> np.ndarray:
    phi = np.array(phi, dtype=np.float64, order="C")
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    _ls_check(lib().orc_ls_advect(ctypes.byref(c), _p(phi), _p(vel), float(dt_), int(nsteps)))
    return phi


def ls_reinit_rhs(c: Config, phi: np.ndarray, phi0: np.ndarray, threshold: float = 5e-2) -> np.ndarray:
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    out = np.zeros_like(phi)
    _ls_check(lib().orc_ls_reinit_rhs(ctypes.byref(c), _p(phi), _p(phi0), float(threshold), _p(out)))
    return out


def ls_reinit(c: Config, phi: np.ndarray, steps: int = 10, threshold: float = 5e-2) -> np.ndarray:
    phi = np.array(phi, dtype=np.float64, order="C")
    _ls_check(lib().orc_ls_reinit(ctypes.byref(c), _p(phi), int(steps), float(threshold)))
    return phi


def ls_weno3_hj(v5, h: float):
    v = np.ascontiguousarray(v5, dtype=np.float64)
    dm, dp = ctypes.c_double(), ctypes.c_double()
    lib().orc_ls_weno3_hj(_p(v), float(h), ctypes.byref(dm), ctypes.byref(dp))
    return dm.value, dp.value


def ls_count_flops(c: Config, phi: np.ndarray, vel: np.ndarray) -> dict:
    """Flops of the level-set functions on this field (totals over the grid;
    the stage combinations per cell)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    vel = np.ascontiguousarray(vel, dtype=np.float64)
    out = np.zeros(5)
    _ls_check(lib().orc_ls_count_flops(ctypes.byref(c), _p(phi), _p(vel), _p(out)))
    return {"geometry": out[0], "advect_rhs": out[1], "reinit_rhs": out[2], "rk3_stage_per_cell": out[3],
            "rk2_stage_per_cell": out[4]}


def ls_interface_riemann(Z1, un1, p1, Z2, un2, p2):
    """(u_Gamma . n, p_Gamma) of the linearised interface Riemann problem."""
    a = np.array([Z1, un1, p1, Z2, un2, p2], dtype=np.float64)
    ug, pg = ctypes.c_double(), ctypes.c_double()
    lib().orc_ls_interface_riemann(_p(a), ctypes.byref(ug), ctypes.byref(pg))
    return ug.value, pg.value


def ls_interface_quantities(c: Config, phi, W1, W2, gamma=(1.4, 1.4), pinf=(0.0, 0.0)):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    W1 = np.ascontiguousarray(W1, dtype=np.float64)
    W2 = np.ascontiguousarray(W2, dtype=np.float64)
    g = np.array(gamma, dtype=np.float64)
    pi = np.array(pinf, dtype=np.float64)
    ug = np.zeros((c.ndim,) + phi.shape)
    pg = np.zeros(phi.shape)
    _ls_check(lib().orc_ls_interface_quantities(ctypes.byref(c), _p(phi), _p(W1), _p(W2), _p(g), _p(pi),
                                                _p(ug), _p(pg)))
    return ug, pg


def ls_extend(c: Config, phi, q, mode: int, steps: int):
    """q: (nq,) + phi.shape, extended in place of a copy and returned."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    q = np.array(q, dtype=np.float64, order="C")
    nq = q.shape[0] if q.ndim == phi.ndim + 1 else 1
    _ls_check(lib().orc_ls_extend(ctypes.byref(c), _p(phi), _p(q), int(nq), int(mode), int(steps)))
    return q


def ls_cut_rhs(c: Config, phi, W, phase: int, ug, pg):
    """d(alpha U)/dt of phase 1 or 2 (c: the phase's single-phase config)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    ug = np.ascontiguousarray(ug, dtype=np.float64)
    pg = np.ascontiguousarray(pg, dtype=np.float64)
    dU = np.zeros_like(W)
    _ls_check(lib().orc_ls_cut_rhs(ctypes.byref(c), _p(phi), _p(W), int(phase), _p(ug), _p(pg), _p(dU)))
    return dU


def ls_mix(c: Config, aU, a0, a1, np_, amix: float = 0.6):
    """Conservative mixing of one phase's volume-weighted state (a copy)."""
    aU = np.array(aU, dtype=np.float64, order="C")
    a0 = np.ascontiguousarray(a0, dtype=np.float64)
    a1 = np.ascontiguousarray(a1, dtype=np.float64)
    np_ = np.ascontiguousarray(np_, dtype=np.float64)
    _ls_check(lib().orc_ls_mix(ctypes.byref(c), int(aU.shape[0]), _p(a0), _p(a1), _p(np_), float(amix), _p(aU)))
    return aU


def ls_init(c1: Config, c2: Config, phi, W1, W2):
    """dict(phi, W1, W2, aU1, aU2, ug, pg) of the level-set model's state."""
    phi = np.array(phi, dtype=np.float64, order="C")
    W1 = np.array(W1, dtype=np.float64, order="C")
    W2 = np.array(W2, dtype=np.float64, order="C")
    aU1, aU2 = np.zeros_like(W1), np.zeros_like(W2)
    ug = np.zeros((c1.ndim,) + phi.shape)
    pg = np.zeros(phi.shape)
    _ls_check(lib().orc_ls_init(ctypes.byref(c1), ctypes.byref(c2), _p(phi), _p(W1), _p(W2), _p(aU1), _p(aU2),
                                _p(ug), _p(pg)))
    return {"phi": phi, "W1": W1, "W2": W2, "aU1": aU1, "aU2": aU2, "ug": ug, "pg": pg}


def ls_step(c1: Config, c2: Config, st: dict, dt: float, nsteps: int, amix: float = 0.6) -> dict:
    """nsteps level-set model steps on a copy of the state dict."""
    st = {k: np.array(v, dtype=np.float64, order="C") for k, v in st.items()}
    _ls_check(lib().orc_ls_step(ctypes.byref(c1), ctypes.byref(c2), float(dt), int(nsteps), float(amix),
                                _p(st["phi"]), _p(st["aU1"]), _p(st["aU2"]), _p(st["W1"]), _p(st["W2"]),
                                _p(st["ug"]), _p(st["pg"])))
    return st
