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
              fixed_dt=case["fixed_dt"], t_end=case["t_end"], eps=eps)
    kw.update(over)
    return oracle.make_config(**kw)
