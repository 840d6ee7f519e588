"""The full benchmark workload -- the 128^3 Taylor-Green vortex over its 500
steps, through the same graph-captured jxf_step the benchmark times --
checked by properties that hold at any size (the oracle needs minutes for
this run; its element-by-element comparison is the 128^3 right-hand side in
test_gpu_parity.py and the 32^3 run over the same 500 steps):

- discrete conservation of mass, momentum and energy on the periodic box;
- the TGV's mirror symmetries x -> 2 pi - x (u odd) and y -> 2 pi - y
  (v odd), which the scheme preserves;
- mixed FP32 against the FP64 run, per field (stated error).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2402_05193_gb300 as jxf  # noqa: E402
from case_tools import momentum_slice, rel_linf  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402

STEPS = 500


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
        s1, _, _ = s.stats()
        out[prec] = (s.state().double().cpu().numpy(), s0, s1, t)
        s.close()
    return out


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


def test_fp64_conservation_and_mirror_symmetry(runs):
    U, s0, s1, t = runs["fp64"]
    cons, sx, sy = _checks(U, s0, s1)
    print("TGV 128^3 x 500 steps FP64: conservation", cons, "mirror x", sx, "mirror y", sy)
    assert cons.max() < 1e-12
    assert max(sx.max(), sy.max()) < 1e-11


def test_fp32_against_fp64(runs):
    U64, _, _, t64 = runs["fp64"]
    U32, s0, s1, t32 = runs["fp32"]
    err = rel_linf(U32, U64)
    mom = momentum_slice(wl.tgv(8))  # momentum components on one shared scale
    err[mom] = np.abs(U32[mom] - U64[mom]).max(axis=(1, 2, 3)) / np.abs(U64[mom]).max()
    cons, sx, sy = _checks(U32, s0, s1)
    print("TGV 128^3 x 500 steps FP32 vs FP64 per field:", err, "conservation", cons,
          "mirror", sx, sy)
    assert abs(t32 / t64 - 1) < 1e-5
    assert err.max() < 1e-3
    assert cons.max() < 1e-4
