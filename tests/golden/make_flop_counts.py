"""Write tests/golden/flop_counts.json: algorithmic flops per cell of the
benchmark workloads, counted by the oracle's instrumented scalar type
(add/sub/mul/div/sqrt = 1 flop, comparisons/min/max/abs/negation = 0).

Counts are taken on the initial state of each workload at a reduced grid
(the per-cell figure of a periodic / uniform-stencil problem does not depend
on the grid size beyond the data-dependent HLLC branch at s* = 0) and are
stated per interior cell; the level-set workload is counted at its benchmark
size (its geometry's cost follows the number of cut cells).  Calls only
``oracle``.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from case_tools import _BC, oracle_config  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402


def count(case, dt=0.0):
    c = oracle_config(case)
    U = oracle.prim_to_cons(c, case["W"])
    f = oracle.count_flops(c, U, dt)
    stage = (f["face_x"] + f["face_y"] + f["face_z"] + f["divergence"] + f["rk_stage"] +
             f["cons2prim"] + f["interface_normal"])
    f["per_stage"] = stage
    f["per_step"] = 3 * stage + f["cfl"]
    return {k: float(v) for k, v in f.items()}


def count_levelset(case, reinit_steps=10):
    """Per cell: the level-set geometry, one advection right-hand side, one
    reinitialisation right-hand side, and one step = one TVD-RK3 advection
    step + reinit_steps second-order reinitialisation steps + the geometry."""
    n = case["n"]
    c = oracle.ls_config(ndim=3, n=n, h=case["h"], bc=[(_BC[a], _BC[b]) for a, b in case["bc"]])
    f = oracle.ls_count_flops(c, case["phi"], case["vel"])
    ncell = n[0] * n[1] * n[2]
    per = {"geometry": f["geometry"] / ncell, "advect_rhs": f["advect_rhs"] / ncell,
           "reinit_rhs": f["reinit_rhs"] / ncell, "rk3_stage": f["rk3_stage_per_cell"],
           "rk2_stage": f["rk2_stage_per_cell"]}
    per["reinit_stage"] = per["reinit_rhs"] + per["rk2_stage"]
    per["per_step"] = (per["geometry"] + 3 * (per["advect_rhs"] + per["rk3_stage"]) +
                       2 * reinit_steps * per["reinit_stage"])
    return {k: float(v) for k, v in per.items()}


def count_levelset_faces(n=32):
    """Per face: the cut-cell right-hand side's face flux of one phase
    (WENO5-JS characteristic reconstruction + HLLC, inviscid, 3-D), counted
    as the single-phase face sweeps on the two-phase drop's ideal-gas phase
    (uniform flow) on a periodic n^3 grid, where every axis has as many
    faces as cells."""
    case = wl.levelset_drop(n)
    g, pi = case["mat2"]
    bc = [(oracle.PERIODIC, oracle.PERIODIC)] * 3
    c = oracle.make_config(ndim=3, n=case["n"], dx=[case["h"]] * 3, bc=bc, gamma=(g, g), pinf=(pi, pi),
                           recon=oracle.CHAR)
    f = oracle.count_flops(c, oracle.prim_to_cons(c, case["W2"]), 0.0)
    return {"face_x": float(f["face_x"]), "face_y": float(f["face_y"]), "face_z": float(f["face_z"])}


def main():
    out = {
        "source": "oracle.count_flops on the initial state; see make_flop_counts.py",
        "tgv_32": count(wl.tgv(32)),
        "tgv_32_weno5z": count(dict(wl.tgv(32), weno="z")),
        "tgv_32_teno6a_visc6": count(dict(wl.tgv(32), weno="teno6a", visc_order=6)),
        "shock_bubble_64x32x32": count(wl.shock_bubble(64, 32, 32), dt=1e-7),
        "shock_bubble_thinc_64x32x32": count(dict(wl.shock_bubble(64, 32, 32), thinc=True), dt=1e-7),
        # the batched drops: a 128^2 drop of the seeded batch's parameter ranges
        # (radius 0.115, centre (0.5, 0.5), Mach 1.8), limiters on
        "drop_128": count(wl.drop(128, 0.115, 0.5, 0.5, 1.8), dt=1e-7),
        # the differentiable Kelvin-Helmholtz workload's forward step
        "kh_256": count(wl.kelvin_helmholtz(256)),
        # the level-set transport workload at its benchmark size
        "levelset_sphere_128": count_levelset(wl.levelset_sphere(128)),
        # the level-set step's cut-cell face fluxes (per face)
        "levelset_drop_faces": count_levelset_faces(),
    }
    path = os.path.join(HERE, "flop_counts.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print(json.dumps(out, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
