"""The full-size three-dimensional shock-bubble workload (256 x 128 x 128
cells, five-equation model, characteristic WENO5-JS, interpolation and flux
limiters, CFL 0.4; §5.3.3 set-up) through the same graph-captured
``jxf_step`` the benchmark times, against the oracle run on the whole grid.

- FP64: every conservative field within 1e-10 (relative L-infinity) of the
  oracle after 100 steps, the same time and the same limiter counts; the
  reported conservation sums against the FP64 sums of the same state.
- FP32 (float bulk, double dt / sums): the per-field error against the FP64
  oracle after the same 100 steps (maximum norm, momentum components on one
  shared scale, and mean), stated and bounded; partial densities stay
  positive and the volume fraction inside [0, 1].
- The workload's full 1000 steps: the FP32 run against the FP64 GPU run
  (itself held to the oracle above), per field in the maximum norm and in
  the mean, stated; both runs admissible throughout.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2402_05193_gb300 as jxf  # noqa: E402
from case_tools import exact_sums, momentum_slice, oracle_config, rel_linf, sum_scale  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402

STEPS = 100
FULL = 1000


@pytest.fixture(scope="module")
def ref():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    case = wl.shock_bubble()
    c = oracle_config(case)
    U, t, k, dl, cnt = oracle.run(c, oracle.prim_to_cons(c, case["W"]), STEPS)
    assert k == STEPS
    return case, c, U, t, cnt


def _gpu(case, precision, steps):
    s = jxf.Solver(case, precision)
    s.set_primitive(case["W"])
    t = s.step(steps)
    U = s.state().double().cpu().numpy()
    W = s.primitive().double().cpu().numpy()
    sums, _, lim = s.stats()
    s.close()
    return U, W, t, lim, sums


def _admissible(W):
    assert np.all(W[0] >= 0) and np.all(W[1] >= 0)
    assert np.all(W[6] >= 0) and np.all(W[6] <= 1)


def test_full_size_fp64_parity(ref):
    case, c, Ur, tr, cnt = ref
    U, _, t, lim, sums = _gpu(case, "fp64", STEPS)
    err = rel_linf(U, Ur)
    print("shock-bubble 256x128x128, %d steps, FP64 per-field rel Linf:" % STEPS, err,
          "limited (IL sides, FL faces):", lim, "oracle:", cnt)
    assert abs(t - tr) <= 1e-12 * tr
    assert err.max() < 1e-10
    assert lim == cnt
    own = np.abs(sums - exact_sums(case, U)) / sum_scale(case, U)
    print("FP64 sums vs the correctly rounded FP64 sum of the same state:", own)
    assert own.max() < 1e-13


def test_full_size_fp32_error(ref):
    case, c, Ur, tr, _ = ref
    U, W, t, _, _ = _gpu(case, "fp32", STEPS)
    err = rel_linf(U, Ur)
    # momentum components share one scale (the transverse ones are ~0 here)
    mom = momentum_slice(case)
    scale = np.max(np.abs(Ur[mom]))
    err[mom] = np.max(np.abs(U[mom] - Ur[mom]), axis=(1, 2, 3)) / scale
    mean = np.mean(np.abs(U - Ur), axis=(1, 2, 3)) / np.mean(np.abs(Ur), axis=(1, 2, 3))
    mean[mom] = np.mean(np.abs(U[mom] - Ur[mom]), axis=(1, 2, 3)) / np.mean(np.abs(Ur[mom]))
    print("shock-bubble 256x128x128, %d steps, FP32 vs FP64 oracle: per-field rel Linf %s, "
          "mean |dU| / mean |U| %s" % (STEPS, err, mean))
    assert abs(t / tr - 1) < 1e-5
    _admissible(W)
    # the maximum sits in cells at the shock and interface fronts
    assert err.max() < 5e-3 and mean.max() < 1e-4


def test_full_length_fp32_against_fp64():
    """All 1000 steps of the workload: the shock has crossed the bubble and
    rolled it up, so a shock or interface displaced by a fraction of a cell
    shows as an O(1) pointwise difference in a few cells; the mean error per
    field measures the bulk."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    case = wl.shock_bubble()
    U64, W64, t64, lim64, _ = _gpu(case, "fp64", FULL)
    U32, W32, t32, lim32, _ = _gpu(case, "fp32", FULL)
    _admissible(W64)
    _admissible(W32)
    mom = momentum_slice(case)
    linf = rel_linf(U32, U64)
    linf[mom] = np.max(np.abs(U32[mom] - U64[mom]), axis=(1, 2, 3)) / np.max(np.abs(U64[mom]))
    mean = np.mean(np.abs(U32 - U64), axis=(1, 2, 3)) / np.mean(np.abs(U64), axis=(1, 2, 3))
    mean[mom] = np.mean(np.abs(U32[mom] - U64[mom]), axis=(1, 2, 3)) / np.mean(np.abs(U64[mom]))
    print("shock-bubble 256x128x128, %d steps, FP32 vs FP64 GPU: t %.9g / %.9g; per-field rel "
          "Linf %s; per-field mean |dU| / mean |U| %s; limited FP64 %s, FP32 %s"
          % (FULL, t32, t64, linf, mean, lim64, lim32))
    assert abs(t32 / t64 - 1) < 1e-4
    assert mean.max() < 1e-2
