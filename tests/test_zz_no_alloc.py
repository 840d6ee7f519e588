"""The allocation-free right-hand side, jxf_rhs_static.

Some callers cannot allocate device memory (another runtime owns the GPU's
memory pool, cudaFree's implicit device synchronisation is not acceptable,
or allocation is forbidden after start-up).  jxf_rhs_static serves them from
a fixed scratch array inside the library; this file checks, through the C
interface, that it returns what jxf_rhs returns bit for bit, on two calls
in a row (the second call must not see the first call's leftovers), and that
it rejects grids whose intermediates exceed the scratch.  It is collected last so that a
run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2402_05193_gb300 as jxf  # noqa: E402
from case_tools import rhs_update_err  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402

PREC = {"fp64": torch.float64, "fp32": torch.float32}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _cases():
    return {
        "spm_char_visc_3d": (lambda seed: wl.smooth_random(3, [20, 16, 12], "spm", seed=seed, viscous=True,
                                                           mu=2e-2), "fp64"),
        "dim_char_lim_2d_water_air": (lambda seed: wl.smooth_random(
            2, [40, 30], "dim", seed=seed, limiter=True, gamma=(6.12, 1.4), pinf=(3.43e8, 0.0),
            rho=(1000.0, 1.2), p0=1e5, u0=30.0), "fp64"),
        "spm_comp_3d_fp32": (lambda seed: wl.smooth_random(3, [24, 20, 16], "spm", seed=seed,
                                                           recon="comp"), "fp32"),
        "spm_char_visc6_3d": (lambda seed: dict(wl.smooth_random(3, [20, 16, 12], "spm", seed=seed,
                                                                viscous=True, mu=2e-2), visc_order=6),
                              "fp64"),
        "dim_char_lim_thinc_3d": (lambda seed: dict(wl.smooth_random(
            3, [16, 12, 10], "dim", seed=seed, limiter=True, gamma=(1.4, 1.66)), thinc=True), "fp64"),
        "spm_char_teno6a_visc6_3d": (lambda seed: dict(wl.smooth_random(
            3, [20, 16, 12], "spm", seed=seed, viscous=True, mu=2e-2), weno="teno6a", visc_order=6), "fp64"),
        "spm_char_teno6a_visc6_3d_fp32": (lambda seed: dict(wl.smooth_random(
            3, [20, 16, 12], "spm", seed=seed, viscous=True, mu=2e-2), weno="teno6a", visc_order=6), "fp32"),
    }


def _state(case, prec):
    """Conservative state of the case in storage precision (device tensor),
    produced by the library's own primitive -> conservative conversion."""
    s = jxf.Solver(case, prec)
    s.set_primitive(case["W"])
    U = s.state()
    s.close()
    return U


@pytest.mark.parametrize("name", list(_cases()))
def test_static_rhs_matches_jxf_rhs_on_two_calls(name):
    make, prec = _cases()[name]
    dt = 1e-7
    for seed in (11, 12):  # two calls in a row with different states
        case = make(seed)
        U = _state(case, prec)
        s = jxf.Solver(case, prec)
        R_ref = s.rhs(U, dt)
        s.close()
        g, e, sc = jxf.structs_from_case(case, prec)
        dU = torch.full_like(U, float("nan"))
        jxf.jxf_rhs_static(g, e, sc, U, dU, dt)
        torch.cuda.synchronize()
        # the same kernels on the same input as jxf_rhs: equal bit for bit
        # (the update-scaled difference is printed when they are not)
        got, ref = dU.cpu().numpy(), R_ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = rhs_update_err(got, ref, U.double().cpu().numpy(), 1e-3)
        assert np.array_equal(got, ref), (name, seed, err)


def test_static_rhs_rejects_oversized_grid_and_host_memory():
    case = wl.tgv(64)  # 64^3 FP64 intermediates exceed the scratch
    g, e, sc = jxf.structs_from_case(case, "fp64")
    U = torch.zeros((5, 64, 64, 64), dtype=torch.float64, device="cuda")
    dU = torch.zeros_like(U)
    with pytest.raises(jxf.JxfError) as ex:
        jxf.jxf_rhs_static(g, e, sc, U, dU, 0.0)
    assert ex.value.status == jxf.JXF_ERR_ARG and "scratch bytes" in str(ex.value)
    small = wl.smooth_random(3, [8, 8, 8], "spm", seed=1)
    g, e, sc = jxf.structs_from_case(small, "fp64")
    Uh = np.zeros((5, 8, 8, 8))
    dUd = torch.zeros((5, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(jxf.JxfError) as ex:
        jxf.jxf_rhs_static(g, e, sc, Uh, dUd, 0.0)
    assert ex.value.status == jxf.JXF_ERR_ARG and "device memory" in str(ex.value)
