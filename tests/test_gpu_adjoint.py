"""Hand-written reverse mode against the oracle's forward tangent and against
central finite differences.

- Tiny grids: the oracle's full Jacobian (one dual-number tangent per unit
  direction) transposed and applied to random cotangents, compared element
  by element with jxf_rhs_vjp.
- Dot-product tests: <v, J d> from the oracle tangent equals <J^T v, d> from
  the GPU adjoint, for one right-hand side and for several RK3 steps.
- Kelvin-Helmholtz: the gradient of the final kinetic energy with respect to
  the initial density (velocity and pressure held fixed) through the
  checkpointed rollout, against central differences of GPU forward runs.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2402_05193_gb300 as jxf  # noqa: E402
from case_tools import oracle_config  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402
from paper_2402_05193_gb300.autograd import rollout  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


TINY = {
    "2d_comp_periodic": dict(ndim=2, n=[6, 5], recon="comp", bc="periodic"),
    "2d_char_periodic": dict(ndim=2, n=[6, 5], recon="char", bc="periodic"),
    "1d_char_zerograd": dict(ndim=1, n=[9], recon="char", bc="zerograd"),
    "2d_char_symmetry": dict(ndim=2, n=[5, 6], recon="char", bc="symmetry"),
    "3d_char_periodic": dict(ndim=3, n=[4, 4, 3], recon="char", bc="periodic"),
    "z_2d_comp_periodic": dict(ndim=2, n=[6, 5], recon="comp", bc="periodic", weno="z"),
    # WENO5-Z: tau = |beta_0 - beta_2| has a kink where beta_0 = beta_2 (e.g. a
    # Fourier mode at the grid's Nyquist frequency, k = 3 on 6 cells); the
    # grids are chosen so that no stencil sits on one
    "z_2d_char_symmetry": dict(ndim=2, n=[5, 7], recon="char", bc="symmetry", weno="z"),
}


@pytest.mark.parametrize("name", list(TINY))
def test_rhs_vjp_equals_transposed_oracle_jacobian(name):
    t = TINY[name]
    case = wl.smooth_random(t["ndim"], t["n"], "spm", seed=21, recon=t["recon"], bc=t["bc"], amp=0.2)
    case["weno"] = t.get("weno", "js")
    c = oracle_config(case)
    U = oracle.prim_to_cons(c, case["W"])
    N = U.size
    J = np.empty((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        _, Rd = oracle.rhs_tangent(c, U, e.reshape(U.shape))
        J[:, k] = Rd.ravel()
    s = jxf.Solver(case, "fp64")
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.normal(size=U.shape)
        g = s.rhs_vjp(_dev(U), _dev(v)).cpu().numpy().ravel()
        ref = J.T @ v.ravel()
        assert np.max(np.abs(g - ref)) <= 1e-11 * np.max(np.abs(ref)), name
    s.close()


@pytest.mark.parametrize("ndim,n,recon,weno", [(2, [24, 20], "char", "js"), (2, [32, 16], "comp", "js"),
                                               (3, [10, 8, 6], "char", "js"),
                                               (2, [24, 20], "char", "z"), (3, [10, 8, 6], "comp", "z")])
def test_rhs_vjp_dot_product(ndim, n, recon, weno):
    case = dict(wl.smooth_random(ndim, n, "spm", seed=5, recon=recon), weno=weno)
    c = oracle_config(case)
    U = oracle.prim_to_cons(c, case["W"])
    rng = np.random.default_rng(9)
    d = rng.normal(size=U.shape) * np.max(np.abs(U), axis=(1, 2, 3), keepdims=True)
    v = rng.normal(size=U.shape)
    _, Jd = oracle.rhs_tangent(c, U, d)
    s = jxf.Solver(case, "fp64")
    JTv = s.rhs_vjp(_dev(U), _dev(v)).cpu().numpy()
    s.close()
    lhs, rhs = np.sum(v * Jd), np.sum(JTv * d)
    scale = np.sum(np.abs(v * Jd))
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


def _fixed_dt_case(case, cfl=0.5):
    c = oracle_config(case)
    dt = oracle.dt(c, oracle.prim_to_cons(c, case["W"]))
    fixed = dict(case)
    fixed["fixed_dt"] = dt
    fixed["t_end"] = 0.0
    return fixed, dt


@pytest.mark.parametrize("recon,weno", [("comp", "js"), ("char", "js"), ("char", "z")])
def test_step_vjp_dot_product_over_steps(recon, weno):
    base = wl.kelvin_helmholtz(24)
    base["recon"] = recon
    base["weno"] = weno
    case, dt = _fixed_dt_case(base)
    nsteps = 6
    c = oracle_config(case)
    U0 = oracle.prim_to_cons(c, case["W"])
    rng = np.random.default_rng(4)
    d = rng.normal(size=U0.shape) * np.max(np.abs(U0), axis=(1, 2, 3), keepdims=True) * 1e-2
    v = rng.normal(size=U0.shape)
    _, Ud = oracle.run_tangent(c, U0, d, nsteps, dt)
    s = jxf.Solver(case, "fp64")
    states = []
    s.set_state(_dev(U0))
    for _ in range(nsteps):
        states.append(s.state())
        s.step(1)
    Ub = _dev(v)
    for k in reversed(range(nsteps)):
        Ub = s.step_vjp(states[k], dt, Ub)
    s.close()
    lhs, rhs = np.sum(v * Ud), np.sum(Ub.cpu().numpy() * d)
    scale = np.sum(np.abs(v * Ud))
    assert abs(lhs - rhs) <= 1e-11 * scale, (lhs, rhs)


def _kinetic_energy(U, vol):
    rho, mx, my = U[0], U[1], U[2]
    return 0.5 * torch.sum((mx * mx + my * my) / rho) * vol


def _kh_gradient(case, dt, nsteps, ckpt, precision="fp64"):
    """dJ/drho0 (u, v, p fixed) through the rollout, and J."""
    s = jxf.Solver(case, precision)
    s.set_primitive(case["W"])
    U0 = s.state().clone().requires_grad_(True)
    UT = rollout(U0, s, nsteps, dt, ckpt)
    vol = case["dx"][0] * case["dx"][1]
    J = _kinetic_energy(UT.double(), vol)
    J.backward()
    Ub = U0.grad.double()
    W = torch.from_numpy(case["W"]).cuda()
    u, v = W[1], W[2]
    g = Ub[0] + u * Ub[1] + v * Ub[2] + 0.5 * (u * u + v * v) * Ub[3]
    s.close()
    return g.cpu().numpy(), float(J)


def _kh_energy(case, dt, nsteps, rho0):
    W = case["W"].copy()
    W[0] = rho0
    s = jxf.Solver(case, "fp64")
    s.set_primitive(W)
    s.step(nsteps)
    U = s.state()
    s.close()
    return float(_kinetic_energy(U, case["dx"][0] * case["dx"][1]))


def test_kh_gradient_against_central_differences():
    base = wl.kelvin_helmholtz(48)
    case, dt = _fixed_dt_case(base)
    nsteps, ckpt = 60, 16  # several checkpoint segments, the last one ragged
    g, J = _kh_gradient(case, dt, nsteps, ckpt)
    rho0 = case["W"][0]
    rng = np.random.default_rng(11)
    dirs = []
    for _ in range(16):
        d = rng.normal(size=rho0.shape)
        dirs.append(d / np.max(np.abs(d)))
    # step size from a sweep on the first direction: smallest disagreement
    errs = {}
    for h in (1e-3, 1e-4, 1e-5, 1e-6):
        fd = (_kh_energy(case, dt, nsteps, rho0 + h * dirs[0]) -
              _kh_energy(case, dt, nsteps, rho0 - h * dirs[0])) / (2 * h)
        errs[h] = abs(fd - np.sum(g * dirs[0])) / abs(fd)
    h = min(errs, key=errs.get)
    worst = 0.0
    for d in dirs:
        fd = (_kh_energy(case, dt, nsteps, rho0 + h * d) - _kh_energy(case, dt, nsteps, rho0 - h * d)) / (2 * h)
        worst = max(worst, abs(fd - np.sum(g * d)) / abs(fd))
    print("KH 48^2, %d steps: FD step %.0e, sweep %s, worst rel err %.2e" % (nsteps, h, errs, worst))
    assert worst < 1e-6


def test_kh_fp32_gradient_error_vs_fp64():
    base = wl.kelvin_helmholtz(48)
    case, dt = _fixed_dt_case(base)
    g64, _ = _kh_gradient(case, dt, 40, 16, "fp64")
    g32, _ = _kh_gradient(case, dt, 40, 16, "fp32")
    rel = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    print("KH 48^2, 40 steps: FP32 gradient relative L2 error vs FP64 %.2e" % rel)
    assert rel < 1e-3


def test_vjp_rejects_unsupported_models():
    case = wl.smooth_random(2, [8, 8], "dim", seed=1)
    s = jxf.Solver(case, "fp64")
    U = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(jxf.JxfError) as ex:
        s.rhs_vjp(U, U)
    assert ex.value.status == jxf.JXF_ERR_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("bc", ["periodic", "zerograd", "symmetry"])
def test_reverse_mode_is_reproducible_bit_for_bit(prec, bc):
    """The stencil adjoints are gathered cell by cell in a fixed order (no
    atomic scatter): two evaluations of the same vector-Jacobian products
    give the same bits, for the right-hand side and for an RK3 step, with
    every kind of boundary (the ends of each line collect several slots)."""
    case, dt = _fixed_dt_case(wl.smooth_random(2, [40, 28], "spm", seed=5, bc=bc, recon="char"))
    s = jxf.Solver(case, prec)
    s.set_primitive(case["W"])
    U = s.state()
    rng = np.random.default_rng(3)
    Rb = _dev(rng.standard_normal(tuple(U.shape))).to(U.dtype)
    outs = []
    for _ in range(2):
        a = torch.empty_like(U)
        jxf.jxf_rhs_vjp(s.h, U, Rb, a, 0.0)
        b = s.step_vjp(U, dt, Rb)
        torch.cuda.synchronize()
        outs.append((a.cpu().numpy(), b.cpu().numpy()))
    s.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
