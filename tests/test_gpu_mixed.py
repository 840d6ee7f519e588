"""Mixed precision (float storage and bulk arithmetic; double dt, sums and,
with p_inf != 0, the recovered pressure) against the FP64 oracle.  The error
is a property of the precision, not a parity bar: each test states the bound
it holds and prints the per-field errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2402_05193_gb300 as jxf  # noqa: E402
from case_tools import (exact_sums, momentum_slice, oracle_config, rel_linf,  # noqa: E402
                        rhs_update_err, sum_scale)
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _compare(case, steps, eps32=True):
    s = jxf.Solver(case, "fp32")
    s.set_primitive(case["W"])
    t = s.step(steps)
    U = s.state().double().cpu().numpy()
    s.close()
    c = oracle_config(case)
    Ur, tr, k, _, _ = oracle.run(c, oracle.prim_to_cons(c, case["W"]), steps)
    return rel_linf(U, Ur), t, tr


@pytest.mark.parametrize("weno", ["js", "z", "teno6a"])
def test_tgv_fp32_error_vs_fp64_oracle(weno):
    err, t, tr = _compare(dict(wl.tgv(32), weno=weno), 100)
    print("TGV 32^3 (%s), 100 steps, FP32 per-field rel Linf:" % weno.upper(), err)
    assert abs(t / tr - 1) < 1e-5
    assert err.max() < (5e-4 if weno == "teno6a" else 1e-4)  # TENO6-A measured 1.7e-4


@pytest.mark.parametrize("thinc", [False, True])
def test_shock_bubble_fp32_error_vs_fp64_oracle(thinc):
    # THINC: bubble off the grid's mirror planes (no round-off-decided ties)
    off = (0.31, 0.17, 0.23) if thinc else (0.0, 0.0, 0.0)
    err, t, tr = _compare(dict(wl.shock_bubble(32, 16, 16, offset=off), thinc=thinc), 30)
    print("shock-bubble 32x16x16%s, 30 steps, FP32 per-field rel Linf:" % (" THINC" if thinc else ""), err)
    assert err.max() < 1e-3


@pytest.mark.parametrize("recon", ["comp", "char"])
def test_teno6a_fp32_cuts_the_stencils_at_a_pascal_scale_jump(recon):
    """FP32 TENO6-A on dimensional data: a 2e5 | 1e5 Pa step (density 2.4 |
    1.2) makes tau6 about 1e10 while the flat sub-stencils have beta = 0, so
    tau6/(beta + 1e-30) is far outside the float range.  The float selection
    must still cut exactly the stencils that cross the jump: its right-hand
    side agrees with the FP64 oracle's (which cuts them) to float round-off,
    where keeping all four stencils across the jump puts the sixth-order
    linear value there and misses by the size of the jump."""
    n = 64
    case = dict(wl.sod(n), recon=recon, weno="teno6a")
    x = (np.arange(n) + 0.5) / n
    W = np.zeros((3, 1, 1, n))
    W[0, 0, 0] = np.where(x < 0.5, 2.4, 1.2)
    W[2, 0, 0] = np.where(x < 0.5, 2e5, 1e5)
    case["W"] = W
    s = jxf.Solver(case, "fp32")
    s.set_primitive(W)
    U = s.state()
    R = s.rhs(U, 0.0).double().cpu().numpy()
    s.close()
    U64 = U.double().cpu().numpy()
    c = oracle_config(case)
    Rr, _ = oracle.rhs(c, U64, 0.0)
    dt = oracle.dt(c, U64)
    err = rhs_update_err(R, Rr, U64, dt, mom=momentum_slice(case))
    print("TENO6-A FP32 (%s) at a 1e5 Pa jump, update-scaled RHS error:" % recon, err)
    assert np.all(np.isfinite(R))
    assert err.max() < 1e-5, err


@pytest.mark.parametrize("weno", ["js", "teno6a"])
def test_air_water_tube_fp32_runs_admissible(weno):
    case = dict(wl.two_material_tube("air_water"), weno=weno)
    s = jxf.Solver(case, "fp32")
    s.set_primitive(case["W"])
    t = s.step(10000)
    W = s.primitive().double().cpu().numpy()
    s.close()
    assert abs(t - case["t_end"]) < 1e-9
    assert np.all(W[0] > 0) and np.all(W[1] > 0)
    c = oracle_config(case)
    Ur, tr, k, _, _ = oracle.run(c, oracle.prim_to_cons(c, case["W"]), 10000)
    Wr = oracle.cons_to_prim(c, Ur)
    err = rel_linf(W, Wr)
    print("air-water tube (%s) FP32 per-field rel Linf (primitives):" % weno.upper(), err)
    assert err.max() < 0.05  # shock positions agree to a cell


def _water_air_states(n=4096, seed=21):
    """Seeded primitive states of the five-equation water (gamma 6.12, p_inf
    3.43e8) / air (gamma 1.4) model on a 1-D row: volume fraction over
    [0, 1] (both ends included), water density 900-1100, air 0.5-5,
    pressure log-uniform over 1e4-1e9 Pa, velocity -500..500 m/s."""
    rng = np.random.default_rng(seed)
    a1 = rng.uniform(0.0, 1.0, n)
    a1[:4] = (1e-8, 1.0 - 1e-8, 1e-4, 1.0 - 1e-4)
    W = np.zeros((5, 1, 1, n))
    W[0, 0, 0] = a1 * rng.uniform(900.0, 1100.0, n)
    W[1, 0, 0] = (1.0 - a1) * rng.uniform(0.5, 5.0, n)
    W[2, 0, 0] = rng.uniform(-500.0, 500.0, n)
    W[3, 0, 0] = 10.0 ** rng.uniform(4.0, 9.0, n)
    W[4, 0, 0] = a1
    case = dict(wl.two_material_tube("air_water", n), W=W)
    return case


def test_float_pressure_against_fp64_evaluation_of_the_same_floats():
    """The float path recovers p = (rho e - B)/A of stiffened-gas states from
    the stored float conservative state in compensated float arithmetic
    (B and A as float pairs, the kinetic energy as a pair, the two large
    differences as exact two-sums), so that neither the cancellation of E
    against B (4.1e8 for water) nor that against up to 1e8 of kinetic
    energy costs accuracy.  Against the FP64 evaluation of the very same
    float inputs (the oracle's conversion) it must agree to a few float
    ulps of p, over volume fractions 0..1, water/air densities, 1e4-1e9 Pa
    and velocities up to 500 m/s (a plain float evaluation misses by
    roundings of E, B and the kinetic energy, printed beside it)."""
    case = _water_air_states()
    s = jxf.Solver(case, "fp32")
    s.set_primitive(case["W"])
    U = s.state().double().cpu().numpy()
    Wf = s.primitive().double().cpu().numpy()
    s.close()
    c = oracle_config(case)
    W64 = oracle.cons_to_prim(c, U)
    g, pi = case["gamma"], case["pinf"]
    a1 = U[4]
    A = a1 / (g[0] - 1) + (1 - a1) / (g[1] - 1)
    B = a1 * g[0] * pi[0] / (g[0] - 1) + (1 - a1) * g[1] * pi[1] / (g[1] - 1)
    ke = 0.5 * U[2] ** 2 / (U[0] + U[1])
    u32 = 2.0 ** -24
    p64, pf = W64[3], Wf[3]
    ulp = np.spacing(np.abs(p64).astype(np.float32)).astype(np.float64)
    d_ulp = np.abs(pf - p64) / ulp
    plain = u32 * (np.abs(U[3]) + B + ke) / A / ulp  # roundings of E, B, ke in a plain float evaluation
    print("float p vs FP64 evaluation of the same floats: max %.2f ulp(p), median %.2f ulp; a plain "
          "float evaluation's rounding of E, B and rho|u|^2/2 alone: median %.3g ulp, max %.3g ulp"
          % (d_ulp.max(), np.median(d_ulp), np.median(plain), plain.max()))
    assert d_ulp.max() <= 4.0, d_ulp.max()
    # velocities (one reciprocal approximation and a product) and the
    # copied partial densities and volume fraction
    for k in (0, 1, 2, 4):
        assert np.all(np.abs(Wf[k] - W64[k]) <= 4 * u32 * np.abs(W64[k])), k


@pytest.mark.parametrize("which", ["tgv128", "water_air"])
def test_float_warp_sums_against_fp64_sums_of_the_stored_floats(which):
    """Conservation sums of a float state: compensated float pairs within
    each warp, then double.  Against the oracle's serial FP64 sum of the
    same stored floats, relative to sum |U| dV (momentum sums cancel)."""
    case = wl.tgv(128) if which == "tgv128" else dict(
        wl.smooth_random(2, [256, 192], "dim", seed=4, limiter=True, gamma=(6.12, 1.4),
                         pinf=(3.43e8, 0.0), rho=(1000.0, 1.2), p0=1e5, u0=30.0))
    s = jxf.Solver(case, "fp32")
    s.set_primitive(case["W"])
    U = s.state().double().cpu().numpy()
    sums, _, _ = s.stats()
    s.close()
    c = oracle_config(case)
    exact = exact_sums(case, U)
    scale = sum_scale(case, U)
    err = np.abs(sums - exact) / scale
    orc = np.abs(oracle.sums(c, U) - exact) / scale
    print("FP32 conservation sums (%s) vs the correctly rounded FP64 sum of the stored floats:" % which,
          err, "(the oracle's serial FP64 sum:", orc, ")")
    assert err.max() < 1e-13


def test_float_sound_speed_through_the_cfl_time_step():
    """rho c^2 of float stiffened-gas states enters the CFL rate; the first
    step's dt (reduced in double from float rates) against the oracle's dt
    of the same float state."""
    case = wl.smooth_random(2, [96, 64], "dim", seed=4, limiter=True, gamma=(6.12, 1.4),
                            pinf=(3.43e8, 0.0), rho=(1000.0, 1.2), p0=1e5, u0=30.0)
    s = jxf.Solver(case, "fp32")
    s.set_primitive(case["W"])
    U = s.state().double().cpu().numpy()
    s.step(1)
    _, dt, _ = s.stats()
    s.close()
    dtr = oracle.dt(oracle_config(case), U)
    print("FP32 CFL dt of a water-air state: %.9g against %.9g (rel %.2e)" % (dt, dtr, abs(dt / dtr - 1)))
    assert abs(dt / dtr - 1) < 1e-6
