"""Helpers turning a workload dict into an oracle configuration (tests only)."""
import oracle

_BC = {"periodic": oracle.PERIODIC, "zerograd": oracle.ZEROGRAD, "symmetry": oracle.SYMMETRY}


def oracle_config(case, eps=None, **over):
    kw = dict(ndim=case["ndim"], n=case["n"], dx=case["dx"],
              bc=[(_BC[a], _BC[b]) for a, b in case["bc"]],
              model=oracle.DIM if case["model"] == "dim" else oracle.SPM,
              gamma=case["gamma"], pinf=case["pinf"], mu=case["mu"], Pr=case["Pr"],
              R=case["R"], recon=oracle.CHAR if case["recon"] == "char" else oracle.COMP,
              viscous=case["viscous"], limiter=case["limiter"], cfl=case["cfl"],
              fixed_dt=case["fixed_dt"], t_end=case["t_end"], eps=eps,
              weno=case.get("weno", "js"), thinc=case.get("thinc", False),
              visc_order=case.get("visc_order", 4))
    kw.update(over)
    return oracle.make_config(**kw)


def rel_linf(a, b):
    """Per-field maximum of |a - b| normalised by max |b| of that field."""
    import numpy as np
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    axes = tuple(range(1, b.ndim))
    scale = np.max(np.abs(b), axis=axes, keepdims=True)
    scale = np.where(scale > 0, scale, 1.0)
    return np.max(np.abs(a - b) / scale, axis=axes).ravel()


def rhs_update_err(R, R_ref, U, dt, mom=None):
    """Per-field error of a right-hand side as it enters one explicit update:
    max |R - R_ref| * dt / max(max |U|, max |dt R_ref|) (R is a small
    difference of large face fluxes, so normalising by max |R| would measure
    cancellation, not the implementation; the second term covers fields that
    start at zero).  ``mom`` = slice of the momentum components, which share
    one scale (components of one vector)."""
    import numpy as np
    R = np.asarray(R, dtype=np.float64)
    axes = tuple(range(1, R.ndim))
    scale = np.maximum(np.max(np.abs(U), axis=axes), np.max(np.abs(R_ref), axis=axes) * dt)
    if mom is not None:
        scale[mom] = np.max(scale[mom])
    return np.max(np.abs(R - R_ref), axis=axes) * dt / np.where(scale > 0, scale, 1.0)


def momentum_slice(case):
    """Indices of the momentum components of a workload's state."""
    first = 2 if case["model"] == "dim" else 1
    return slice(first, first + case["ndim"])


def exact_sums(case, U):
    """Per-variable sum of U over the cells times the cell volume, correctly
    rounded (math.fsum): the reference for the library's conservation sums,
    free of the summation-order error of a serial double sum."""
    import math

    import numpy as np
    vol = float(np.prod(case["dx"]))
    return np.array([math.fsum((np.asarray(u, dtype=np.float64) * vol).ravel()) for u in U])


def sum_scale(case, U):
    """Per-variable sum of |U| dV (the scale of a sum whose terms cancel, such
    as the TGV's zero total momentum); 1 for fields that are zero."""
    import numpy as np
    s = exact_sums(case, np.abs(U))
    return np.where(s > 0, s, 1.0)
