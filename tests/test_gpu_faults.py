"""Failure detection without a GPU fault: non-admissible or non-finite
states are caught by the device status word and reported as
JXF_ERR_NONPHYSICAL by the next synchronising call; invalid arguments are
rejected before any launch; the context stays usable afterwards."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2402_05193_gb300 as jxf  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("inject", ["negative_density", "nan_pressure", "negative_pressure"])
def test_injected_state_reports_nonphysical(precision, inject):
    case = wl.smooth_random(2, [16, 12], "spm", seed=2)
    W = case["W"].copy()
    if inject == "negative_density":
        W[0, 0, 5, 7] = -0.3
    elif inject == "nan_pressure":
        W[3, 0, 2, 2] = np.nan
    else:
        W[3, 0, 9, 1] = -50.0  # rho c^2 < 0
    s = jxf.Solver(case, precision)
    s.set_primitive(W)
    with pytest.raises(jxf.JxfError) as ex:
        s.step(1)
    assert ex.value.status == jxf.JXF_ERR_NONPHYSICAL
    # the handle and the context stay usable: a good state runs again
    s.set_primitive(case["W"])
    t = s.step(2)
    assert t > 0
    s.close()
    torch.cuda.synchronize()


def test_invalid_arguments_are_rejected_before_launch():
    case = wl.sod(32)
    s = jxf.Solver(case, "fp64")
    s.set_primitive(case["W"])
    with pytest.raises(jxf.JxfError) as ex:
        s.step(-1)
    assert ex.value.status == jxf.JXF_ERR_ARG
    with pytest.raises(jxf.JxfError) as ex:
        jxf.jxf_rhs(s.h, np.zeros(3), np.zeros(3), -1.0)
    assert ex.value.status == jxf.JXF_ERR_ARG
    with pytest.raises(jxf.JxfError) as ex:
        jxf.jxf_set_time(s.h, float("nan"))
    assert ex.value.status == jxf.JXF_ERR_ARG
    assert s.step(5) > 0
    s.close()


def test_batch_reports_the_failing_simulation():
    cases = wl.drop_batch(nsim=3, seed=4, sizes=(24, 32))
    bad = 1
    cases[bad]["W"] = cases[bad]["W"].copy()
    cases[bad]["W"][0, 0, 3, 3] = -1.0
    B = jxf.Batch(cases, "fp64")
    B.set_primitives()
    B.step(2)
    for k in range(3):
        if k == bad:
            with pytest.raises(jxf.JxfError):
                B.stats(k)
        else:
            B.stats(k)
    B.close()


def test_allocation_failures_are_reported_and_leave_nothing_behind():
    """An allocation failure (injected on the host at every allocation of
    handle creation in turn, and at a call's first use of its scratch) is
    reported as JXF_ERR_OOM, frees what was allocated and leaves a handle
    that was already created usable."""
    case = wl.tgv(96)
    g, e, sc = jxf.structs_from_case(case, "fp64")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(40):
        jxf.jxf_fail_allocation_after(k)
        try:
            h = jxf.jxf_create(g, e, sc)
        except jxf.JxfError as ex:
            assert ex.status == jxf.JXF_ERR_OOM
            failures += 1
            continue
        finally:
            jxf.jxf_fail_allocation_after(-1)
        jxf.jxf_destroy(h)
        break
    assert failures >= 10  # every allocation of the handle failed once before one succeeded
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < 32 << 20  # nothing left behind
    s = jxf.Solver(case, "fp64")
    s.set_primitive(case["W"])
    U = s.state()
    jxf.jxf_fail_allocation_after(0)
    with pytest.raises(jxf.JxfError) as ex:
        s.rhs(U)  # the right-hand side's scratch
    jxf.jxf_fail_allocation_after(-1)
    assert ex.value.status == jxf.JXF_ERR_OOM
    R = s.rhs(U)  # usable afterwards
    assert torch.isfinite(R).all()
    s.step(2)
    s.close()
