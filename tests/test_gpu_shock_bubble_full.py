"""The full-size three-dimensional shock-bubble workload (256 x 128 x 128
cells, five-equation model, characteristic WENO5-JS, interpolation and flux
limiters, CFL 0.4; §5.3.3 set-up) through the same graph-captured
``jxf_step`` the benchmark times, against the oracle run on the whole grid.

- FP64: every conservative field within 1e-10 (relative L-infinity) of the
  oracle after 10 steps, the same time and the same limiter counts.
- FP32 (float bulk, double dt / sums): the per-field error against the FP64
  oracle (momentum components on one shared scale) is stated and bounded;
  partial densities stay positive and the volume fraction inside [0, 1].
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2402_05193_gb300 as jxf  # noqa: E402
from case_tools import momentum_slice, oracle_config, rel_linf  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402

STEPS = 10


@pytest.fixture(scope="module")
def ref():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    case = wl.shock_bubble()
    c = oracle_config(case)
    U, t, k, dl, cnt = oracle.run(c, oracle.prim_to_cons(c, case["W"]), STEPS)
    assert k == STEPS
    return case, U, t, cnt


def _gpu(case, precision):
    s = jxf.Solver(case, precision)
    s.set_primitive(case["W"])
    t = s.step(STEPS)
    U = s.state().double().cpu().numpy()
    W = s.primitive().double().cpu().numpy()
    _, _, lim = s.stats()
    s.close()
    return U, W, t, lim


def test_full_size_fp64_parity(ref):
    case, Ur, tr, cnt = ref
    U, _, t, lim = _gpu(case, "fp64")
    err = rel_linf(U, Ur)
    print("shock-bubble 256x128x128, %d steps, FP64 per-field rel Linf:" % STEPS, err,
          "limited (IL sides, FL faces):", lim)
    assert abs(t - tr) <= 1e-12 * tr
    assert err.max() < 1e-10
    assert lim == cnt


def test_full_size_fp32_error(ref):
    case, Ur, tr, _ = ref
    U, W, t, _ = _gpu(case, "fp32")
    err = rel_linf(U, Ur)
    # momentum components share one scale (the transverse ones are ~0 here)
    mom = momentum_slice(case)
    scale = np.max(np.abs(Ur[mom]))
    err[mom] = np.max(np.abs(U[mom] - Ur[mom]), axis=(1, 2, 3)) / scale
    print("shock-bubble 256x128x128, %d steps, FP32 per-field rel Linf vs FP64 oracle:" % STEPS, err)
    assert abs(t / tr - 1) < 1e-5
    assert np.all(W[0] >= 0) and np.all(W[1] >= 0)
    assert np.all(W[6] >= 0) and np.all(W[6] <= 1)
    assert err.max() < 1e-3
