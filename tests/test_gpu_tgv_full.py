"""The full benchmark workload -- the 128^3 Taylor-Green vortex over its 500
steps, through the same graph-captured jxf_step the benchmark times:

- FP64 against the oracle run over the same 500 steps on the whole grid,
  element by element: every conservative field within 1e-10 (relative
  L-infinity), the same time and last dt;
- the conservation sums the library reports (FP64, reduced on the device)
  against the FP64 sums of its own final state and of the oracle's;
- discrete conservation of mass, momentum and energy on the periodic box;
- the TGV's mirror symmetries x -> 2 pi - x (u odd) and y -> 2 pi - y
  (v odd), which the scheme preserves;
- mixed FP32 against the FP64 oracle, per field (stated error).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2402_05193_gb300 as jxf  # noqa: E402
from case_tools import exact_sums, momentum_slice, oracle_config, rel_linf, sum_scale  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402

STEPS = 500
TOL64 = 1e-10


@pytest.fixture(scope="module")
def runs():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    out = {}
    for prec in ("fp64", "fp32"):
        case = wl.tgv(128)
        s = jxf.Solver(case, prec)
        s.set_primitive(case["W"])
        s0, _, _ = s.stats()
        t = s.step(STEPS)
        s1, dt_last, _ = s.stats()
        out[prec] = (s.state().double().cpu().numpy(), s0, s1, t, dt_last)
        s.close()
    return out


@pytest.fixture(scope="module")
def ref():
    case = wl.tgv(128)
    c = oracle_config(case)
    U, t, k, dt_last, _ = oracle.run(c, oracle.prim_to_cons(c, case["W"]), STEPS)
    assert k == STEPS
    return c, U, t, dt_last


def _checks(U, s0, s1):
    scale = np.abs(U).reshape(U.shape[0], -1).max(axis=1)
    vol = (2 * np.pi) ** 3
    cons = np.abs(s1 - s0) / np.maximum(np.abs(s0), scale * vol)
    mx = U[..., ::-1].copy()
    mx[1] *= -1
    my = U[:, :, ::-1, :].copy()
    my[2] *= -1
    sx = np.abs(mx - U).reshape(U.shape[0], -1).max(axis=1) / scale
    sy = np.abs(my - U).reshape(U.shape[0], -1).max(axis=1) / scale
    return cons, sx, sy


def test_fp64_500_steps_against_the_oracle(runs, ref):
    U, _, s1, t, dt_last = runs["fp64"]
    c, Ur, tr, dtr = ref
    err = rel_linf(U, Ur)
    print("TGV 128^3 x 500 steps FP64 vs oracle, per-field rel Linf:", err,
          "t %.17g / %.17g, last dt %.17g / %.17g" % (t, tr, dt_last, dtr))
    assert abs(t - tr) <= 1e-12 * tr
    assert abs(dt_last - dtr) <= 1e-12 * dtr
    assert err.max() < TOL64, err


def test_fp64_conservation_sums_against_fp64_sums(runs, ref):
    """The device's per-block FP64 partials, folded in a fixed order, against
    the correctly rounded FP64 sum of the same final state (summation order
    only), and against the sums of the oracle's own state (parity level)."""
    U, _, s1, _, _ = runs["fp64"]
    c, Ur, _, _ = ref
    case = wl.tgv(128)
    scale = sum_scale(case, U)
    own = np.abs(s1 - exact_sums(case, U)) / scale
    orc = np.abs(s1 - exact_sums(case, Ur)) / scale
    print("TGV 128^3 FP64 sums: vs FP64 sum of the same state", own, "vs the oracle's state", orc)
    assert own.max() < 1e-13
    assert orc.max() < TOL64


def test_fp64_conservation_and_mirror_symmetry(runs):
    U, s0, s1, t, _ = runs["fp64"]
    cons, sx, sy = _checks(U, s0, s1)
    print("TGV 128^3 x 500 steps FP64: conservation", cons, "mirror x", sx, "mirror y", sy)
    assert cons.max() < 1e-12
    assert max(sx.max(), sy.max()) < 1e-11


def test_fp32_against_the_fp64_oracle(runs, ref):
    U32, s0, s1, t32, _ = runs["fp32"]
    c, Ur, tr, _ = ref
    err = rel_linf(U32, Ur)
    mom = momentum_slice(wl.tgv(8))  # momentum components on one shared scale
    err[mom] = np.abs(U32[mom] - Ur[mom]).max(axis=(1, 2, 3)) / np.abs(Ur[mom]).max()
    cons, sx, sy = _checks(U32, s0, s1)
    print("TGV 128^3 x 500 steps FP32 vs FP64 oracle per field:", err, "conservation", cons,
          "mirror", sx, sy)
    assert abs(t32 / tr - 1) < 1e-5
    assert err.max() < 1e-3
    assert cons.max() < 1e-4
