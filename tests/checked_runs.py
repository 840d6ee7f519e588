"""Small runs of every kernel family (whole grids in both precisions, the
fused float sweep, limiters, THINC, TENO6-A, boundary kinds, 1-D/2-D/3-D,
blocks of a decomposed grid, the batch, reverse mode, the allocation-free
right-hand side), used to compare the index-checked build of the library
(JXF_LIB pointing at it) with the release build.  Run as a script it writes
the results to an .npz file; a bounds violation raises (JXF_ERR_BOUNDS)."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _grid_cases(wl):
    return {
        "tgv16": (wl.tgv(16), 10),
        "tgv16_teno6a_visc6": (dict(wl.tgv(16), weno="teno6a", visc_order=6), 4),
        "bubble_thinc": (dict(wl.shock_bubble(16, 12, 8, offset=(0.31, 0.17, 0.23)), thinc=True), 8),
        "sym_zerograd": (dict(wl.smooth_random(3, [12, 10, 9], "spm", seed=3, recon="comp"),
                              bc=[("symmetry", "zerograd"), ("zerograd", "symmetry"),
                                  ("symmetry", "zerograd")]), 8),
        "sod64": (wl.sod(64), 40),
        "kh32": (wl.kelvin_helmholtz(32, steps=10), 10),
    }


def run(out_path):
    import torch

    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    from paper_2402_05193_gb300.decomp import SlabGrid
    torch.cuda.set_device(0)
    res = {}
    for name, (case, steps) in _grid_cases(wl).items():
        for prec in ("fp64", "fp32"):
            s = jxf.Solver(case, prec)
            s.set_primitive(case["W"])
            s.step(steps)
            res["%s_%s" % (name, prec)] = s.state().double().cpu().numpy()
            s.close()
    for name, case, nb in (("tgv16_blocks", wl.tgv(16), 2), ("bubble_blocks", wl.shock_bubble(16, 12, 8), 2)):
        for prec in ("fp64", "fp32"):
            g = SlabGrid(case, prec, nb)
            g.set_primitive(case["W"])
            g.step(6)
            res["%s_%s" % (name, prec)] = g.state().double().cpu().numpy()
            g.stats()
            g.close()
    drops = [wl.drop(N, 0.12, 0.5, 0.5, 1.8) for N in (32, 48, 64)]
    B = jxf.Batch(drops, "fp32")
    B.set_primitives()
    B.step(5)
    for k in range(len(drops)):
        res["batch_%d" % k] = B.state(k).double().cpu().numpy()
        B.stats(k)
    B.close()
    case = wl.smooth_random(2, [20, 14], "spm", seed=5, bc="symmetry", recon="char")
    s = jxf.Solver(dict(case, fixed_dt=1e-4, t_end=0.0), "fp64")
    s.set_primitive(case["W"])
    U = s.state()
    Rb = torch.from_numpy(np.random.default_rng(3).standard_normal(tuple(U.shape))).cuda()
    res["step_vjp"] = s.step_vjp(U, 1e-4, Rb).cpu().numpy()
    s.close()
    small = wl.smooth_random(3, [10, 9, 8], "spm", seed=2, viscous=True, mu=2e-2)
    s = jxf.Solver(small, "fp64")
    s.set_primitive(small["W"])
    U = s.state()
    s.close()
    g_, e_, sc_ = jxf.structs_from_case(small, "fp64")
    dU = torch.empty_like(U)
    jxf.jxf_rhs_static(g_, e_, sc_, U, dU, 1e-6)
    torch.cuda.synchronize()
    res["static_rhs"] = dU.cpu().numpy()
    np.savez(out_path, **res)


if __name__ == "__main__":
    run(sys.argv[1])
