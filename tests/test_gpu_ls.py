"""The level-set kernels (§3.5, App. D) against the oracle, through the C
interface: interface geometry (apertures, volume fraction, interface
segment, normal), the advection right-hand side and TVD-RK3 steps, the
reinitialisation right-hand side and its pseudo-time steps, the interface
quantities of the cut cells and the three extensions.  Grids of
several sizes (a ragged last block) and every boundary condition; FP64
parity at 1e-12 (the vertex values, and so every sign decision of the
apertures, are the same sums in the same order on both sides)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as orc  # noqa: E402
import paper_2402_05193_gb300 as jxf  # noqa: E402

P, Z, S = orc.PERIODIC, orc.ZEROGRAD, orc.SYMMETRY


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _field(kind, ndim, n, h, seed):
    rng = np.random.default_rng(seed)
    axes = [(np.arange(n[e]) + 0.5) * h for e in range(ndim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]  # X, Y(, Z), arrays of shape (n_z,) n_y, n_x
    L = [n[e] * h for e in range(ndim)]
    if kind == "sphere":
        c = [0.5 * L[e] + rng.uniform(-0.1, 0.1) * L[e] for e in range(ndim)]
        R = 0.3 * min(L)
        return R - np.sqrt(sum((grids[e] - c[e]) ** 2 for e in range(ndim)))
    # smooth periodic bumps: many cut cells of every sign pattern
    phi = np.full(grids[0].shape, 0.1)
    for _ in range(3):
        k = rng.integers(1, 3, size=ndim)
        ph = rng.uniform(0, 2 * math.pi, size=ndim)
        term = np.ones_like(phi)
        for e in range(ndim):
            term = term * np.cos(2 * math.pi * k[e] * grids[e] / L[e] + ph[e])
        phi = phi + rng.uniform(0.3, 0.6) * term
    return phi


CASES = {
    "sphere3_zerograd_20": (3, [20, 20, 20], [(Z, Z)] * 3, "sphere"),
    "bumps3_periodic_24x18x20": (3, [24, 18, 20], [(P, P)] * 3, "bumps"),
    "bumps3_mixed_17x13x11": (3, [17, 13, 11], [(S, Z), (P, P), (Z, S)], "bumps"),
    "circle2_symmetry_33x29": (2, [33, 29], [(S, S), (S, Z)], "sphere"),
    "bumps2_periodic_40x24": (2, [40, 24], [(P, P)] * 2, "bumps"),
}


def _setup(name, seed=0):
    ndim, n, bc, kind = CASES[name]
    h = 1.0 / 16
    phi = _field(kind, ndim, n, h, seed)
    cfg = orc.ls_config(ndim=ndim, n=n, h=h, bc=bc)
    grid = jxf.ls_grid(ndim, n, h, bc)
    return ndim, n, h, phi, cfg, grid


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_geometry_matches_the_oracle(name):
    ndim, n, h, phi, cfg, grid = _setup(name)
    ap_o, al_o, dg_o, nr_o = orc.ls_geometry(cfg, phi)
    nf = jxf.jxf_ls_nface(grid)
    assert nf == ap_o.size
    ap = torch.zeros(nf, dtype=torch.float64, device="cuda")
    al = torch.zeros(phi.shape, dtype=torch.float64, device="cuda")
    dg = torch.zeros_like(al)
    nr = torch.zeros((ndim,) + phi.shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_geometry(grid, _dev(phi), ap, al, dg, nr)
    torch.cuda.synchronize()
    e = [np.abs(ap.cpu().numpy() - ap_o).max(), np.abs(al.cpu().numpy() - al_o).max(),
         np.abs(dg.cpu().numpy() - dg_o).max() / h ** (ndim - 1), np.abs(nr.cpu().numpy() - nr_o).max()]
    cut = int(((al_o > 0) & (al_o < 1)).sum())
    print("%s: %d cut cells, max |diff| apertures %.2g, alpha %.2g, dGamma/h^(d-1) %.2g, normal %.2g"
          % (name, cut, *e))
    assert cut > 20
    assert max(e) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_advection_rhs_and_steps_match_the_oracle(name):
    ndim, n, h, phi, cfg, grid = _setup(name, seed=1)
    rng = np.random.default_rng(2)
    vel = rng.uniform(-1.0, 1.0, size=(ndim,) + phi.shape)  # both signs: both stencils
    r_o = orc.ls_rhs(cfg, phi, vel)
    r = torch.zeros(phi.shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_rhs(grid, _dev(phi), _dev(vel), r)
    scale = np.abs(r_o).max()
    assert np.abs(r.cpu().numpy() - r_o).max() < 1e-12 * scale
    dt = 0.2 * h
    out_o = orc.ls_advect(cfg, phi, vel, dt, 5)
    p = _dev(phi)
    scratch = torch.zeros((2,) + phi.shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_advect(grid, p, _dev(vel), dt, 5, scratch)
    err = np.abs(p.cpu().numpy() - out_o).max() / np.abs(out_o).max()
    print("%s: advection RHS and 5 RK3 steps, max rel diff %.2g" % (name, err))
    assert err < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_reinitialisation_matches_the_oracle(name):
    ndim, n, h, phi, cfg, grid = _setup(name, seed=3)
    phi = phi * (1.0 + 0.8 * np.sin(7.0 * phi))  # same zero set, |grad phi| far from 1
    r_o = orc.ls_reinit_rhs(cfg, phi, phi, 5e-2)
    r = torch.zeros(phi.shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_reinit_rhs(grid, _dev(phi), _dev(phi), 5e-2, r)
    assert np.abs(r.cpu().numpy() - r_o).max() < 1e-12
    out_o = orc.ls_reinit(cfg, phi, 10, 5e-2)
    p = _dev(phi)
    scratch = torch.zeros((2,) + phi.shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_reinit(grid, p, 10, 5e-2, scratch)
    out = p.cpu().numpy()
    err = np.abs(out - out_o).max()
    changed = int((np.abs(out_o - phi) > 0).sum())
    print("%s: reinitialisation, %d cells changed, max |diff| %.2g" % (name, changed, err))
    assert changed > 20
    assert err < 1e-12


def test_full_size_sphere_geometry_and_transport():
    """The benchmark's 128^3 sphere in a solid-body rotation: geometry and one
    advection + reinitialisation step against the oracle at every cell."""
    n, h = [128, 128, 128], 1.0 / 128
    x = (np.arange(128) + 0.5) * h
    Zg, Yg, Xg = np.meshgrid(x, x, x, indexing="ij")
    phi = 0.25 - np.sqrt((Xg - 0.5) ** 2 + (Yg - 0.6) ** 2 + (Zg - 0.5) ** 2)
    vel = np.stack([-(Yg - 0.5), Xg - 0.5, np.zeros_like(Xg)])
    bc = [(Z, Z)] * 3
    cfg = orc.ls_config(ndim=3, n=n, h=h, bc=bc)
    grid = jxf.ls_grid(3, n, h, bc)
    ap_o, al_o, dg_o, nr_o = orc.ls_geometry(cfg, phi)
    ap = torch.zeros(jxf.jxf_ls_nface(grid), dtype=torch.float64, device="cuda")
    al = torch.zeros(phi.shape, dtype=torch.float64, device="cuda")
    dg, nr = torch.zeros_like(al), torch.zeros((3,) + phi.shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_geometry(grid, _dev(phi), ap, al, dg, nr)
    assert np.abs(ap.cpu().numpy() - ap_o).max() < 1e-12
    assert np.abs(al.cpu().numpy() - al_o).max() < 1e-12
    vol = al.sum().item() * h ** 3
    print("128^3 sphere: volume %.6f (exact %.6f)" % (vol, 4.0 / 3.0 * math.pi * 0.25 ** 3))
    dt = 0.5 * h / 0.5
    ref = orc.ls_reinit(cfg, orc.ls_advect(cfg, phi, vel, dt, 1), 10, 5e-2)
    p = _dev(phi)
    scratch = torch.zeros((2,) + phi.shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_advect(grid, p, _dev(vel), dt, 1, scratch)
    jxf.jxf_ls_reinit(grid, p, 10, 5e-2, scratch)
    assert np.abs(p.cpu().numpy() - ref).max() < 1e-12


def test_invalid_grids_are_rejected():
    phi = torch.zeros(27, dtype=torch.float64, device="cuda")
    out = torch.zeros(200, dtype=torch.float64, device="cuda")
    bad = [jxf.ls_grid(1, [27], 0.1, [(Z, Z)]),                        # 1-D
           jxf.ls_grid(2, [9, 2], 0.1, [(Z, Z), (Z, Z)])]               # fewer than 3 cells
    g = jxf.ls_grid(2, [9, 3], 0.1, [(Z, Z), (Z, Z)])
    g.hi[1] = 0.5                                                       # non-cubic cells
    bad.append(g)
    g = jxf.ls_grid(2, [9, 3], 0.1, [(P, Z), (Z, Z)])                   # one-sided periodic
    bad.append(g)
    for grid in bad:
        with pytest.raises(jxf.JxfError) as ex:
            jxf.jxf_ls_rhs(grid, phi, out, out[:27])
        assert ex.value.status == jxf.JXF_ERR_ARG
        assert jxf.jxf_ls_nface(grid) == -1


def _geometry_dev(grid, phi, ndim):
    ap = torch.zeros(jxf.jxf_ls_nface(grid), dtype=torch.float64, device="cuda")
    al = torch.zeros(phi.shape, dtype=torch.float64, device="cuda")
    dg = torch.zeros_like(al)
    nr = torch.zeros((ndim,) + phi.shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_geometry(grid, _dev(phi), ap, al, dg, nr)
    return al, dg, nr


@pytest.mark.parametrize("name", list(CASES))
def test_interface_quantities_match_the_oracle(name):
    ndim, n, h, phi, cfg, grid = _setup(name, seed=4)
    rng = np.random.default_rng(6)
    shape = phi.shape

    def prim(rho, p):
        u = [0.3 * np.sin(2.0 * phi + k) + rng.uniform(-0.1, 0.1) for k in range(ndim)]
        return np.stack([np.full(shape, rho) * (1.0 + 0.1 * np.cos(3.0 * phi))] + u +
                        [np.full(shape, p) * (1.0 + 0.2 * np.sin(5.0 * phi))])
    W1, W2 = prim(1000.0, 2e5), prim(1.2, 1e5)
    gamma, pinf = (6.12, 1.4), (3.43e8, 0.0)
    ug_o, pg_o = orc.ls_interface_quantities(cfg, phi, W1, W2, gamma, pinf)
    al, dg, nr = _geometry_dev(grid, phi, ndim)
    ug = torch.zeros((ndim,) + shape, dtype=torch.float64, device="cuda")
    pg = torch.zeros(shape, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_interface(grid, _dev(W1), _dev(W2), gamma, pinf, al, dg, nr, ug, pg)
    cut = int((pg_o != 0).sum())
    eu = np.abs(ug.cpu().numpy() - ug_o).max() / max(np.abs(ug_o).max(), 1e-300)
    ep = np.abs(pg.cpu().numpy() - pg_o).max() / np.abs(pg_o).max()
    print("%s: %d cut cells, interface velocity rel diff %.2g, pressure %.2g" % (name, cut, eu, ep))
    assert cut > 20 and eu < 1e-12 and ep < 1e-12


@pytest.mark.parametrize("mode,steps", [(0, 10), (1, 10), (2, 20)])
@pytest.mark.parametrize("name", ["sphere3_zerograd_20", "bumps3_mixed_17x13x11", "circle2_symmetry_33x29"])
def test_extension_matches_the_oracle(name, mode, steps):
    ndim, n, h, phi, cfg, grid = _setup(name, seed=5)
    rng = np.random.default_rng(7 + mode)
    q = rng.normal(size=(3,) + phi.shape)
    ref = orc.ls_extend(cfg, phi, q, mode, steps)
    al, dg, nr = _geometry_dev(grid, phi, ndim)
    qd = _dev(q)
    scratch = torch.zeros_like(qd)
    jxf.jxf_ls_extend(grid, _dev(phi), al, dg, nr, qd, 3, mode, steps, scratch)
    out = qd.cpu().numpy()
    changed = int((np.abs(ref - q) > 0).sum())
    err = np.abs(out - ref).max()
    print("%s: extension mode %d, %d steps, %d values changed, max |diff| %.2g" % (name, mode, steps, changed, err))
    assert changed > 50 and err < 1e-12


@pytest.mark.parametrize("recon", ["comp", "char", "z_char", "teno_char"])
@pytest.mark.parametrize("name", ["sphere3_zerograd_20", "bumps3_periodic_24x18x20", "bumps3_mixed_17x13x11",
                                  "circle2_symmetry_33x29"])
def test_cut_cell_rhs_matches_the_oracle(name, recon):
    ndim, n, h, phi, cfg, grid = _setup(name, seed=8)
    rng = np.random.default_rng(9)
    shape = phi.shape
    ug = 0.3 * rng.normal(size=(ndim,) + shape)
    pg = 1.0 + 0.3 * rng.uniform(size=shape)
    al, _, nr = _geometry_dev(grid, phi, ndim)
    ap = torch.zeros(jxf.jxf_ls_nface(grid), dtype=torch.float64, device="cuda")
    dgd = torch.zeros_like(al)
    jxf.jxf_ls_geometry(grid, _dev(phi), ap, al, dgd, nr)
    bc = CASES[name][2]
    for phase, (gam, pinf) in ((1, (6.12, 20.0)), (2, (1.4, 0.0))):
        ocfg = orc.make_config(ndim=ndim, n=n, dx=[h] * ndim, bc=bc, gamma=(gam, gam), pinf=(pinf, pinf),
                               recon=orc.COMP if recon == "comp" else orc.CHAR,
                               weno={"z_char": "z", "teno_char": "teno6a"}.get(recon, "js"))
        W = np.stack([1.0 + 0.3 * rng.uniform(size=shape)] + [0.4 * rng.normal(size=shape) for _ in range(ndim)] +
                     [1.0 + 0.4 * rng.uniform(size=shape)])
        ref = orc.ls_cut_rhs(ocfg, phi, W, phase, ug, pg)
        eos = jxf.jxf_eos()
        eos.model = jxf.JXF_SPM
        eos.gamma[0], eos.gamma[1] = gam, gam
        eos.pinf[0], eos.pinf[1] = pinf, pinf
        sch = jxf.jxf_scheme()
        sch.recon = {"comp": jxf.JXF_WENO5JS_COMP, "char": jxf.JXF_WENO5JS_CHAR, "z_char": jxf.JXF_WENO5Z_CHAR,
                     "teno_char": jxf.JXF_TENO6A_CHAR}[recon]
        sch.precision = jxf.JXF_FP64
        sch.weno_eps = 1e-6
        dU = torch.zeros(W.shape, dtype=torch.float64, device="cuda")
        scratch = torch.zeros((ndim + 2) * jxf.jxf_ls_nface(grid), dtype=torch.float64, device="cuda")
        jxf.jxf_ls_cut_rhs(grid, eos, sch, ap, dgd, nr, _dev(W), phase, _dev(ug), _dev(pg), dU, scratch)
        got = dU.cpu().numpy()
        scale = np.abs(ref).reshape(ndim + 2, -1).max(axis=1).reshape((-1,) + (1,) * ndim)
        err = np.abs((got - ref) / scale).max()
        print("%s %s phase %d: cut-cell RHS rel diff %.2g" % (name, recon, phase, err))
        assert err < 1e-12


@pytest.mark.parametrize("ndim,n,bc", [(3, [14, 11, 9], P), (3, [10, 9, 8], Z), (2, [33, 21], P), (2, [17, 19], Z)])
def test_mixing_matches_the_oracle(ndim, n, bc):
    rng = np.random.default_rng(70 + ndim)
    shape = tuple(reversed(n))
    a1 = rng.uniform(size=shape)
    a1[a1 < 0.15] = 0.0
    a0 = np.where(rng.uniform(size=shape) < 0.2, 0.0, np.maximum(a1, 0.05))
    nv = ndim + 2
    aU = rng.uniform(0.5, 2.0, size=(nv,) + shape) * np.maximum(a1, 0.02)
    nrm = rng.normal(size=(ndim,) + shape)
    nrm /= np.sqrt((nrm ** 2).sum(axis=0))
    cfg = orc.ls_config(ndim=ndim, n=n, h=0.1, bc=[(bc, bc)] * ndim)
    ref = orc.ls_mix(cfg, aU, a0, a1, nrm, 0.6)
    grid = jxf.ls_grid(ndim, n, 0.1, [(bc, bc)] * ndim)
    ntrg = 7 if ndim == 3 else 3
    out = _dev(aU)
    scratch = torch.zeros((ntrg + 1) * nv * a1.size, dtype=torch.float64, device="cuda")
    jxf.jxf_ls_mix(grid, nv, _dev(a0), _dev(a1), _dev(nrm), 0.6, out, scratch)
    got = out.cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    changed = int((np.abs(ref - aU).max(axis=0) > 0).sum())
    print("mixing %dD %s: %d cells changed, max rel diff %.2g" % (ndim, "periodic" if bc == P else "zero-gradient",
                                                                 changed, err))
    assert changed > 50 and err < 1e-13
    # conservation on the device too
    assert np.all(np.abs(got.reshape(nv, -1).sum(axis=1) - aU.reshape(nv, -1).sum(axis=1))
                  < 1e-13 * np.abs(aU).reshape(nv, -1).sum(axis=1))


# ------------------------------------------------------- the level-set step --
def _phase_eos(gam, pinf):
    eos = jxf.jxf_eos()
    eos.model = jxf.JXF_SPM
    eos.gamma[0], eos.gamma[1] = gam, gam
    eos.pinf[0], eos.pinf[1] = pinf, pinf
    return eos


def _step_scheme(recon=None):
    sch = jxf.jxf_scheme()
    sch.recon = jxf.JXF_WENO5JS_CHAR if recon is None else recon
    sch.precision = jxf.JXF_FP64
    sch.weno_eps = 1e-6
    return sch


def _run_step_pair(ndim, n, h, bc, ph1, ph2, phi, W1, W2, dt, nsteps, weno="js"):
    """The same level-set steps on the oracle and through jxf_ls_init /
    jxf_ls_step (characteristic WENO5 with Jiang-Shu or WENO5-Z weights, or
    TENO6-A);
    returns (oracle state, device state as numpy)."""
    c1, c2 = (orc.make_config(ndim=ndim, n=n, dx=[h] * ndim, bc=bc, gamma=(g, g), pinf=(pi, pi), recon=orc.CHAR,
                              weno=weno) for g, pi in (ph1, ph2))
    ref = orc.ls_step(c1, c2, orc.ls_init(c1, c2, phi, W1, W2), dt, nsteps)
    grid = jxf.ls_grid(ndim, n, h, bc)
    e1, e2 = _phase_eos(*ph1), _phase_eos(*ph2)
    sch = _step_scheme({"js": jxf.JXF_WENO5JS_CHAR, "z": jxf.JXF_WENO5Z_CHAR, "teno6a": jxf.JXF_TENO6A_CHAR}[weno])
    dphi, dW1, dW2 = _dev(phi), _dev(W1), _dev(W2)
    aU1, aU2 = torch.zeros_like(dW1), torch.zeros_like(dW2)
    qg = torch.zeros((ndim + 1,) + phi.shape, dtype=torch.float64, device="cuda")
    work = torch.zeros(jxf.jxf_ls_step_work(grid), dtype=torch.float64, device="cuda")
    jxf.jxf_ls_init(grid, e1, e2, sch, dphi, dW1, dW2, aU1, aU2, qg, work)
    jxf.jxf_ls_step(grid, e1, e2, sch, dt, nsteps, 0.6, dphi, aU1, aU2, dW1, dW2, qg, work)
    torch.cuda.synchronize()
    got = {"phi": dphi.cpu().numpy(), "aU1": aU1.cpu().numpy(), "aU2": aU2.cpu().numpy(), "W1": dW1.cpu().numpy(),
           "W2": dW2.cpu().numpy(), "ug": qg[:ndim].cpu().numpy(), "pg": qg[ndim].cpu().numpy()}
    return ref, got


def _step_errors(ref, got):
    """Largest difference of each field relative to its component's scale
    (a component that vanishes, as the transverse momentum of a 1-D flow,
    is measured against 1e-3 of the field's largest component)."""
    err = {}
    for k in ("phi", "aU1", "aU2", "W1", "W2", "ug", "pg"):
        r, g = ref[k], got[k]
        if r.ndim > ref["phi"].ndim:  # per component scale
            scale = np.abs(r).reshape(r.shape[0], -1).max(axis=1)
            scale = np.maximum(scale, 1e-3 * scale.max())
            err[k] = float((np.abs(g - r).reshape(r.shape[0], -1).max(axis=1) / scale).max())
        else:
            err[k] = float(np.abs(g - r).max() / max(np.abs(r).max(), 1e-300))
    return err


@pytest.mark.parametrize("weno", ["js", "z"])
def test_level_set_step_air_helium_tube_matches_the_oracle(weno):
    """The air-helium shock tube (Sec. 5.3.1) on 200 x 4 cells, the interface
    starting on a cell face, 150 steps to t = 0.15, with Jiang-Shu or the
    paper's default WENO5-Z weights: every field of the state agrees with
    the oracle's to accumulated round-off."""
    N, ny = 200, 4
    h = 1.0 / N
    bc = [(Z, Z), (P, P)]
    x = (np.arange(N) + 0.5) * h
    shape = (ny, N)
    phi = np.broadcast_to(0.5 - x, shape).copy()
    zero = np.zeros(shape)
    W1 = np.stack([np.ones(shape), zero, zero, np.ones(shape)])
    W2 = np.stack([np.full(shape, 0.125), zero, zero, np.full(shape, 0.1)])
    ref, got = _run_step_pair(2, [N, ny], h, bc, (1.4, 0.0), (1.67, 0.0), phi, W1, W2, 0.2 * h, 150, weno=weno)
    err = _step_errors(ref, got)
    print("air-helium tube (%s), 150 steps:" % weno, {k: "%.1e" % v for k, v in err.items()})
    assert max(err.values()) < 1e-9
    # and the device run is the physics: the interface near the exact contact
    row = got["phi"][0]
    i = int(np.argmax(row < 0))
    xg = x[i - 1] + h * row[i - 1] / (row[i - 1] - row[i])
    _, _, _, _, star = orc.exact_riemann((1.4, 0.0, 1.0, 0.0, 1.0), (1.67, 0.0, 0.125, 0.0, 0.1),
                                         np.array([0.0]))
    assert abs(xg - (0.5 + star[1] * 0.15)) < 0.25 * h


def test_level_set_step_air_water_tube_matches_the_oracle():
    """The air-water shock tube (Sec. 5.3.2; water 1000 kg/m^3 at 1e9 Pa,
    p_inf 3.43e8, against air at 1e5 Pa) on 200 x 4 cells, 194 steps to
    t = 1.5e-4 s: every field within accumulated round-off of the oracle
    (the stiffened gas recovers p from E with log10(rho e / (p + p_inf))
    digits lost, here under one)."""
    N, ny, L, x0 = 200, 4, 1.5, 0.8
    h = L / N
    bc = [(Z, Z), (P, P)]
    x = (np.arange(N) + 0.5) * h
    shape = (ny, N)
    phi = np.broadcast_to(x0 - x, shape).copy()
    zero = np.zeros(shape)
    W1 = np.stack([np.full(shape, 1000.0), zero, zero, np.full(shape, 1e9)])
    W2 = np.stack([np.full(shape, 20.0), zero, zero, np.full(shape, 1e5)])
    ref, got = _run_step_pair(2, [N, ny], h, bc, (6.12, 3.43e8), (1.4, 0.0), phi, W1, W2, 1.5e-4 / 194, 194)
    err = _step_errors(ref, got)
    print("air-water tube, 194 steps:", {k: "%.1e" % v for k, v in err.items()})
    assert max(err.values()) < 1e-9


def test_level_set_step_shock_bubble_matches_the_oracle():
    """The air-helium shock-bubble interaction of Sec. 5.3.3 with the
    level-set model, 2-D at half resolution (128 x 64 cells of 1 mm, the
    helium cylinder of radius 12.5 cells a little off the grid's mirror
    lines, the Ma 1.22 shock 15 cells upstream, zero-gradient sides): 60
    steps, the shock through the bubble's front; every field within
    accumulated round-off of the oracle."""
    nx, ny, dx = 128, 64, 1e-3
    R, cx, cy, xs = 12.5 * dx, 50.31 * dx, 32.17 * dx, 35.0 * dx
    x, y = (np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx
    Y, X = np.meshgrid(y, x, indexing="ij")
    phi = R - np.sqrt((X - cx) ** 2 + (Y - cy) ** 2)
    post = X < xs
    zero = np.zeros(phi.shape)
    W1 = np.stack([np.full(phi.shape, 0.1660), zero, zero, np.full(phi.shape, 101325.0)])
    W2 = np.stack([np.where(post, 1.6573, 1.2041), np.where(post, 114.5, 0.0), zero,
                   np.where(post, 159056.0, 101325.0)])
    dt = 0.4 * dx / (114.5 + 1.2 * math.sqrt(1.66 * 159056.0 / 0.166))
    ref, got = _run_step_pair(2, [nx, ny], dx, [(Z, Z), (Z, Z)], (1.66, 0.0), (1.4, 0.0), phi, W1, W2, dt, 60)
    err = _step_errors(ref, got)
    print("shock-bubble, 60 steps:", {k: "%.1e" % v for k, v in err.items()})
    assert max(err.values()) < 1e-9
    assert float(ref["W1"][3].max()) > 1.2e5  # the shock has entered the helium


@pytest.mark.parametrize("case,weno", [("drop2_periodic_32", "js"), ("drop3_mixed_18x16x14", "js"),
                                       ("drop3_mixed_18x16x14", "teno6a")])
def test_level_set_step_moving_drop_matches_the_oracle(case, weno):
    """A stiffened-gas drop in a perturbed gas flow, 2-D periodic or 3-D with
    every boundary kind (WENO5-JS, and TENO6-A in 3-D): a few steps on both
    sides, every field within accumulated round-off; the device totals
    conserve on the periodic grid."""
    rng = np.random.default_rng(91)
    if case.startswith("drop2"):
        ndim, n, bc = 2, [32, 32], [(P, P)] * 2
    else:
        ndim, n, bc = 3, [18, 16, 14], [(S, Z), (P, P), (Z, S)]
    h = 1.0 / 32
    shape = tuple(reversed(n))
    axes = [(np.arange(n[e]) + 0.5) * h for e in range(ndim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
    c = [0.5 * n[e] * h + 0.3 * h for e in range(ndim)]
    phi = 0.12 - np.sqrt(sum((grids[e] - c[e]) ** 2 for e in range(ndim)))
    u = [0.4 + 0.05 * np.sin(2 * np.pi * grids[(e + 1) % ndim]) for e in range(ndim)]
    p = 1.0 + 0.05 * rng.uniform(size=shape)
    W1 = np.stack([np.full(shape, 5.0)] + u + [p])
    W2 = np.stack([np.ones(shape)] + u + [p])
    dt = 0.3 * h / 3.0
    ref, got = _run_step_pair(ndim, n, h, bc, (4.4, 6.0), (1.4, 0.0), phi, W1, W2, dt, 5, weno=weno)
    err = _step_errors(ref, got)
    print("%s (%s), 5 steps:" % (case, weno), {k: "%.1e" % v for k, v in err.items()})
    assert max(err.values()) < 1e-10
    if ndim == 2:
        init = orc.ls_init(*(orc.make_config(ndim=2, n=n, dx=[h] * 2, bc=bc, gamma=(g, g), pinf=(pi, pi))
                             for g, pi in ((4.4, 6.0), (1.4, 0.0))), phi, W1, W2)
        tot0 = init["aU1"].sum(axis=(1, 2)) + init["aU2"].sum(axis=(1, 2))
        tot = got["aU1"].sum(axis=(1, 2)) + got["aU2"].sum(axis=(1, 2))
        assert np.abs((tot - tot0) / tot0).max() < 1e-13


def test_level_set_step_rejects_what_it_does_not_support():
    grid = jxf.ls_grid(3, [8, 8, 8], 0.1, [(P, P)] * 3)
    e1, e2, sch = _phase_eos(1.4, 0.0), _phase_eos(1.67, 0.0), _step_scheme()
    nc = 8 ** 3
    phi = torch.zeros(nc, dtype=torch.float64, device="cuda")
    st = [torch.zeros(5 * nc, dtype=torch.float64, device="cuda") for _ in range(4)]
    qg = torch.zeros(4 * nc, dtype=torch.float64, device="cuda")
    work = torch.zeros(jxf.jxf_ls_step_work(grid), dtype=torch.float64, device="cuda")
    dim = _phase_eos(1.4, 0.0)
    dim.model = jxf.JXF_DIM
    visc = _step_scheme()
    visc.viscous = 1
    v1, v2 = _phase_eos(1.4, 0.0), _phase_eos(1.67, 0.0)
    for e in (v1, v2):  # a valid viscous material
        e.mu, e.Pr, e.R = 1e-3, 0.72, 287.0
    for eos_a, eos_b, scheme in ((dim, e2, sch), (v1, v2, visc)):
        with pytest.raises(jxf.JxfError) as ex:
            jxf.jxf_ls_step(grid, eos_a, eos_b, scheme, 1e-3, 1, 0.6, phi, *st, qg, work)
        assert ex.value.status == jxf.JXF_ERR_UNSUPPORTED
    with pytest.raises(jxf.JxfError) as ex:
        jxf.jxf_ls_step(grid, e1, e2, sch, float("nan"), 1, 0.6, phi, *st, qg, work)
    assert ex.value.status == jxf.JXF_ERR_ARG
    bad = jxf.ls_grid(3, [8, 8, 8], 0.1, [(P, P)] * 3)
    bad.hi[1] = bad.lo[1] + 1.0  # non-cubic cells
    assert jxf.jxf_ls_step_work(grid) > 0
    with pytest.raises(ValueError):
        jxf.jxf_ls_step_work(bad)


def test_level_set_step_at_the_bench_size_conserves():
    """The bench's two-phase drop (128^3 periodic cells) through the same
    calls bench.py times, three steps: the totals of mass, momentum and
    energy over both phases stay to round-off (the cut-cell fluxes, the
    interface force and power and the mixing only move content), the drop
    keeps its volume, the uniform flow stays uniform in the bulk of each
    phase, and the state stays finite."""
    from paper_2402_05193_gb300 import workloads as wl
    case = wl.levelset_drop(128)
    h, dt = case["h"], case["dt"]
    grid = jxf.ls_grid(3, case["n"], h, [(P, P)] * 3)
    phi, W1, W2 = _dev(case["phi"]), _dev(case["W1"]), _dev(case["W2"])
    aU1, aU2 = torch.zeros_like(W1), torch.zeros_like(W2)
    qg = torch.zeros((4,) + tuple(phi.shape), dtype=torch.float64, device="cuda")
    work = torch.zeros(jxf.jxf_ls_step_work(grid), dtype=torch.float64, device="cuda")
    e1, e2, sch = _phase_eos(*case["mat1"]), _phase_eos(*case["mat2"]), _step_scheme()
    jxf.jxf_ls_init(grid, e1, e2, sch, phi, W1, W2, aU1, aU2, qg, work)
    tot0 = (aU1.sum(dim=(1, 2, 3)) + aU2.sum(dim=(1, 2, 3))).cpu().numpy()
    jxf.jxf_ls_step(grid, e1, e2, sch, dt, 3, 0.6, phi, aU1, aU2, W1, W2, qg, work)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(aU1).all() and torch.isfinite(aU2).all() and torch.isfinite(phi).all())
    tot = (aU1.sum(dim=(1, 2, 3)) + aU2.sum(dim=(1, 2, 3))).cpu().numpy()
    rel = np.abs(tot - tot0) / np.abs(tot0)
    print("128^3 drop, 3 steps: relative change of the totals", rel)
    assert rel.max() < 1e-12
    ap = torch.zeros(jxf.jxf_ls_nface(grid), dtype=torch.float64, device="cuda")
    al = torch.zeros_like(phi)
    dg, nr = torch.zeros_like(phi), torch.zeros((3,) + tuple(phi.shape), dtype=torch.float64, device="cuda")
    jxf.jxf_ls_geometry(grid, phi, ap, al, dg, nr)
    vol = float(al.sum()) * h ** 3
    assert abs(vol / (4.0 / 3.0 * math.pi * 0.25 ** 3) - 1.0) < 2e-3
    inside, outside = (al == 1.0), (al == 0.0)
    for W, m in ((W1, inside), (W2, outside)):
        for k, u in enumerate((0.4, 0.3, 0.2)):
            assert float((W[1 + k][m] - u).abs().max()) < 2e-2


def test_level_set_class_runs_the_step_of_the_c_interface():
    """The binding's LevelSet class (state tensors, jxf_ls_init, jxf_ls_step)
    gives the oracle's state on the 3-D drop with WENO5-Z, as the direct
    calls do."""
    from paper_2402_05193_gb300 import workloads as wl
    case = wl.levelset_drop(16)
    bc = [(P, P)] * 3
    c1, c2 = (orc.make_config(ndim=3, n=case["n"], dx=[case["h"]] * 3, bc=bc, gamma=(g, g), pinf=(pi, pi),
                              recon=orc.CHAR, weno="z") for g, pi in (case["mat1"], case["mat2"]))
    ref = orc.ls_step(c1, c2, orc.ls_init(c1, c2, case["phi"], case["W1"], case["W2"]), case["dt"], 4)
    ls = jxf.LevelSet(3, case["n"], case["h"], bc, case["mat1"], case["mat2"], "z_char")
    ls.set_state(case["phi"], case["W1"], case["W2"])
    ls.step(case["dt"], 4)
    torch.cuda.synchronize()
    got = {"phi": ls.phi.cpu().numpy(), "aU1": ls.aU1.cpu().numpy(), "aU2": ls.aU2.cpu().numpy(),
           "W1": ls.W1.cpu().numpy(), "W2": ls.W2.cpu().numpy(), "ug": ls.qg[:3].cpu().numpy(),
           "pg": ls.qg[3].cpu().numpy()}
    err = _step_errors(ref, got)
    print("LevelSet class, 4 steps:", {k: "%.1e" % v for k, v in err.items()})
    assert max(err.values()) < 1e-10
    # the drop's volume (alpha summed) stays that of the initial geometry
    # (which on 16^3 cells is 5 % below the sphere's: a radius of 4 cells)
    _, al0, _, _ = orc.ls_geometry(orc.ls_config(ndim=3, n=case["n"], h=case["h"], bc=bc), case["phi"])
    _, al, _, _ = ls.geometry()
    assert abs(float(al.sum()) / al0.sum() - 1.0) < 1e-3


@pytest.mark.parametrize("phase", [1, 2])
def test_one_phase_everywhere_step_is_the_single_phase_step(phase):
    """A level set of one sign on the whole grid: jxf_ls_step's state of that
    phase equals the single-grid solver's (jxf_step with the same fixed dt,
    characteristic WENO5-JS) after 4 steps to round-off; the two paths share
    the face flux and nothing else."""
    from paper_2402_05193_gb300 import workloads as wl
    rng = np.random.default_rng(60 + phase)
    n, h = [12, 10, 8], 0.1
    sbc = [(wl.PERIODIC, wl.PERIODIC), (wl.ZEROGRAD, wl.SYMMETRY), (wl.SYMMETRY, wl.ZEROGRAD)]
    lbc = [(P, P), (Z, S), (S, Z)]
    mat = (1.4, 0.0) if phase == 1 else (4.4, 6.0)
    shape = (n[2], n[1], n[0])
    W = np.stack([1.0 + 0.2 * rng.uniform(size=shape)] + [0.3 * rng.normal(size=shape) for _ in range(3)] +
                 [1.0 + 0.3 * rng.uniform(size=shape)])
    dt, nst = 0.01, 4
    case = wl._case("one_phase", ndim=3, n=n, dx=[h] * 3, bc=sbc, W=W, gamma=(mat[0], mat[0]),
                    pinf=(mat[1], mat[1]), recon="char", fixed_dt=dt, steps=nst)
    s = jxf.Solver(case, "fp64")
    s.set_primitive(W)
    s.step(nst)
    U_ref = s.state().cpu().numpy()
    s.close()
    ls = jxf.LevelSet(3, n, h, lbc, mat, mat, "js_char")
    ls.set_state(np.full(shape, 0.7 if phase == 1 else -0.7), W, W)
    ls.step(dt, nst)
    aU = (ls.aU1 if phase == 1 else ls.aU2).cpu().numpy()
    scale = np.abs(U_ref).reshape(5, -1).max(axis=1)[:, None, None, None]
    err = np.abs((aU - U_ref.reshape(aU.shape)) / scale).max()
    print("phase %d everywhere: jxf_ls_step vs jxf_step, max rel diff %.2g" % (phase, err))
    assert err < 1e-12
