"""The differentiable Kelvin-Helmholtz workload at full size: 256^2 cells,
2000 fixed-dt RK3 steps, checkpoints every 100 steps.  Gradient of the final
kinetic energy with respect to the initial density through the hand-written
adjoint, against central differences of GPU forward runs on 16 seeded
directions, in FP64; the FP32 gradient's error against it is stated.

Over 2000 steps the roll-up makes the energy's higher derivatives large, so a
central difference needs a small step, where round-off of the forward runs
(amplified by the flow) sets a floor near 1e-7: as in the paper's AD-vs-FD
check, each direction takes the step of smaller error from a sweep."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2402_05193_gb300 as jxf  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402
from paper_2402_05193_gb300.autograd import rollout  # noqa: E402

N, STEPS, CKPT = 256, 2000, 100


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _dt0(case):
    """The CFL 0.5 bound of the initial state (computed on the host from the
    primitive field: CFL / max sum_d (|u_d| + c)/dx_d)."""
    W = case["W"]
    c = np.sqrt(1.4 * W[3] / W[0])
    rate = (np.abs(W[1]) + c) / case["dx"][0] + (np.abs(W[2]) + c) / case["dx"][1]
    return 0.5 / rate.max()


def _energy(U, vol):
    return 0.5 * torch.sum((U[1] * U[1] + U[2] * U[2]) / U[0]) * vol


def _gradient(case, dt, precision):
    s = jxf.Solver(case, precision)
    s.set_primitive(case["W"])
    U0 = s.state().clone().requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    UT = rollout(U0, s, STEPS, dt, CKPT)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    vol = case["dx"][0] * case["dx"][1]
    J = _energy(UT.double(), vol)
    J.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    Ub = U0.grad.double()
    W = torch.from_numpy(case["W"]).cuda()
    u, v = W[1], W[2]
    g = Ub[0] + u * Ub[1] + v * Ub[2] + 0.5 * (u * u + v * v) * Ub[3]
    s.close()
    return g.cpu().numpy(), float(J), t1 - t0, t2 - t1


def test_kh256_gradient_fd_16_directions():
    case = wl.kelvin_helmholtz(N, steps=STEPS)
    dt = _dt0(case)
    case = dict(case, fixed_dt=dt, t_end=0.0)
    g, J, tf, tb = _gradient(case, dt, "fp64")
    s = jxf.Solver(case, "fp64")
    vol = case["dx"][0] * case["dx"][1]

    def energy(rho0):
        W = case["W"].copy()
        W[0] = rho0
        s.set_primitive(W)
        s.step(STEPS)
        return float(_energy(s.state(), vol))

    rho0 = case["W"][0]
    rng = np.random.default_rng(11)
    dirs = [d / np.max(np.abs(d)) for d in (rng.normal(size=rho0.shape) for _ in range(16))]
    def cd(d, h):
        return (energy(rho0 + h * d) - energy(rho0 - h * d)) / (2 * h)

    errs, errs_l1, steps = [], [], []
    for d in dirs:
        adj = np.sum(g * d)
        best = min(((abs(cd(d, h) - adj), h) for h in (1e-5, 1e-6)))
        errs.append(best[0] / abs(adj))                  # relative to the derivative
        errs_l1.append(best[0] / np.sum(np.abs(g * d)))  # relative to its summed terms
        steps.append(best[1])
    h = {k: steps.count(k) for k in set(steps)}
    sweep = {"errors": [float("%.1e" % e) for e in errs], "l1": [float("%.1e" % e) for e in errs_l1]}
    s.close()
    g32, _, tf32, tb32 = _gradient(case, dt, "fp32")
    rel32 = np.linalg.norm(g32 - g) / np.linalg.norm(g)
    print("KH 256^2 x %d steps (ckpt %d): J = %.6e; FP64 forward %.2f s, backward %.2f s; "
          "FD steps chosen %s; per-direction rel err %s (max %.2e, median %.2e); error over "
          "sum |g_i d_i| %s (max %.2e); FP32 forward %.2f s, backward %.2f s, gradient rel L2 "
          "error vs FP64 %.2e"
          % (STEPS, CKPT, J, tf, tb, h, sweep["errors"], max(errs), float(np.median(errs)),
             sweep["l1"], max(errs_l1), tf32, tb32, rel32))
    assert float(np.median(errs)) < 1e-6 and max(errs_l1) < 1e-6
    assert rel32 < 1e-2
