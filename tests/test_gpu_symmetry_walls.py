"""Symmetry walls against the mirrored full domain, on the GPU path in both
precisions.  The Taylor-Green vortex is mirror symmetric about the planes
x, y, z = 0 and pi (the velocity component normal to a plane is odd across
it, the rest even), so the octant [0, pi]^3 with symmetry walls on all six
faces must reproduce the octant of the periodic [0, 2 pi]^3 run (§3.1:
symmetry boundaries mirror the state and flip the normal velocity).  This
drives every mirrored code path of the face sweeps, the viscous flux and the
velocity-gradient pass, including the float sweeps' separate copy for faces
without mirrored cells.  The arithmetic per face is the same either way; only
the instruction scheduling of the compiled copies may differ, hence a bound
at the rounding level of each precision."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2402_05193_gb300 as jxf  # noqa: E402
from case_tools import momentum_slice, rel_linf  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402

N = 32
STEPS = 20


def _run(case, prec):
    s = jxf.Solver(case, prec)
    s.set_primitive(case["W"])
    t = s.step(STEPS)
    U = s.state().double().cpu().numpy()
    s.close()
    return U, t


# (field bound, time bound): float runs agree to a few ulps per step, and
# their dt comes from the float CFL rates of states that differ at that level
@pytest.mark.parametrize("prec,bound,tbound", [("fp64", 1e-12, 1e-12), ("fp32", 1e-5, 1e-6)])
@pytest.mark.parametrize("recon", ["char", "comp"])
def test_tgv_octant_with_symmetry_walls_matches_periodic_box(prec, bound, tbound, recon):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    full = dict(wl.tgv(N), recon=recon)
    h = N // 2
    octant = dict(full, n=[h] * 3, bc=[("symmetry", "symmetry")] * 3,
                  W=np.ascontiguousarray(full["W"][:, :h, :h, :h]))
    Uf, tf = _run(full, prec)
    Uo, to = _run(octant, prec)
    ref = Uf[:, :h, :h, :h]
    err = rel_linf(Uo, ref)
    mom = momentum_slice(full)  # momentum components on one shared scale (w starts at 0)
    err[mom] = np.abs(Uo[mom] - ref[mom]).max(axis=(1, 2, 3)) / np.abs(ref[mom]).max()
    print("TGV octant with symmetry walls vs periodic box, %s %s, %d steps: t %.17g / %.17g, "
          "per-field rel Linf %s" % (prec, recon, STEPS, to, tf, err))
    assert abs(to / tf - 1) < tbound
    assert err.max() < bound
