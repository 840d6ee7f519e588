"""The C interface: the library builds for sm_103a, loads without a GPU and
exports every function include/*.h declares; argument checks that need no
device work."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(jxf_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libjxf():
    from paper_2402_05193_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_interface():
    names = _declared()
    for must in ("jxf_create", "jxf_destroy", "jxf_set_state", "jxf_get_state", "jxf_rhs",
                 "jxf_step", "jxf_stats", "jxf_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libjxf):
    missing = [n for n in _declared() if not hasattr(libjxf, n)]
    assert not missing, missing


def test_null_arguments_are_rejected_without_a_device(libjxf):
    libjxf.jxf_create.restype = ctypes.c_int
    libjxf.jxf_create.argtypes = [ctypes.c_void_p] * 4
    assert libjxf.jxf_create(None, None, None, None) == 1  # JXF_ERR_ARG
    libjxf.jxf_destroy.argtypes = [ctypes.c_void_p]
    libjxf.jxf_destroy.restype = ctypes.c_int
    assert libjxf.jxf_destroy(None) == 1
    libjxf.jxf_last_error.restype = ctypes.c_char_p
    libjxf.jxf_last_error.argtypes = [ctypes.c_void_p]
    assert b"null handle" in libjxf.jxf_last_error(None)


def test_invalid_grids_are_rejected_before_any_device_work(libjxf):
    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    case = wl.sod(8)
    g, e, s = jxf.structs_from_case(case)
    h = ctypes.c_void_p()
    bad = [("ndim", 4), ("n0", 0), ("inactive", 2), ("periodic_small", 2), ("viscous_dim", 1),
           ("recon", 6), ("visc_order", 3), ("thinc", 2), ("thinc_spm", 1), ("faces_2p31", 1290)]
    for what, val in bad:
        g2, e2, s2 = jxf.structs_from_case(case)
        if what == "ndim":
            g2.ndim = val
        elif what == "n0":
            g2.n[0] = val
        elif what == "inactive":
            g2.n[1] = val
        elif what == "periodic_small":
            g2.n[0] = val
            g2.bc[0][0] = g2.bc[0][1] = jxf.JXF_BC_PERIODIC
        elif what == "viscous_dim":
            e2.model = jxf.JXF_DIM
            s2.viscous = 1
        elif what == "recon":
            s2.recon = val
        elif what == "visc_order":
            s2.visc_order = val
        elif what == "thinc":
            e2.model = jxf.JXF_DIM
            s2.thinc = val
        elif what == "thinc_spm":
            s2.thinc = val
        elif what == "faces_2p31":  # 32-bit face indices: more than 2^31 - 1 faces per axis
            g2.ndim = 3
            for k in range(3):
                g2.n[k] = val
                g2.lo[k], g2.hi[k] = 0.0, 1.0
                g2.bc[k][0] = g2.bc[k][1] = jxf.JXF_BC_ZEROGRAD
        rc = jxf.lib().jxf_create(ctypes.byref(g2), ctypes.byref(e2), ctypes.byref(s2), ctypes.byref(h))
        assert rc in (1, 6), (what, rc)
        assert not h.value


def test_static_rhs_checks_the_structs_as_create_does(libjxf):
    """jxf_rhs_static rejects what jxf_create rejects (a viscous order other
    than 2/4/6, a negative or NaN viscosity, ...) before any device work;
    only the time-step requirement is left out."""
    import paper_2402_05193_gb300 as jxf
    from paper_2402_05193_gb300 import workloads as wl
    f = jxf.lib().jxf_rhs_static
    f.argtypes = [ctypes.POINTER(jxf.jxf_grid), ctypes.POINTER(jxf.jxf_eos), ctypes.POINTER(jxf.jxf_scheme),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_char_p, ctypes.c_size_t]
    f.restype = ctypes.c_int
    base = wl.smooth_random(3, [8, 8, 8], "spm", seed=1, viscous=True, mu=1e-2)
    bad = [("visc_order", 3), ("mu", -1.0), ("mu", float("nan")), ("Pr", 0.0), ("R", -1.0),
           ("recon", 6), ("ndim", 4), ("periodic_small", 2), ("thinc_spm", 1)]
    dummy = ctypes.c_void_p(256)  # never dereferenced: the checks come first
    for what, val in bad:
        g, e, s = jxf.structs_from_case(base)
        if what == "visc_order":
            s.visc_order = val
        elif what in ("mu", "Pr", "R"):
            setattr(e, what, val)
        elif what == "recon":
            s.recon = val
        elif what == "ndim":
            g.ndim = val
        elif what == "periodic_small":
            g.n[0] = val
        elif what == "thinc_spm":
            s.thinc = val
        msg = ctypes.create_string_buffer(256)
        rc = f(ctypes.byref(g), ctypes.byref(e), ctypes.byref(s), dummy, dummy, 0.0, None, msg, 256)
        assert rc in (jxf.JXF_ERR_ARG, jxf.JXF_ERR_UNSUPPORTED), (what, rc)
        assert msg.value.startswith(b"jxf_rhs_static:"), (what, msg.value)
    # no CFL number and no fixed dt: accepted by the checks (a bare right-hand
    # side takes no step); what follows needs a device
    g, e, s = jxf.structs_from_case(base)
    s.cfl, s.fixed_dt = 0.0, 0.0
    msg = ctypes.create_string_buffer(256)
    rc = f(ctypes.byref(g), ctypes.byref(e), ctypes.byref(s), dummy, dummy, 0.0, None, msg, 256)
    assert b"invalid grid" not in msg.value, msg.value


def test_level_set_step_rejects_bad_arguments_without_a_device(libjxf):
    """The level-set step checks its grid, materials, scheme and arguments on
    the host before any device work: non-cubic cells, a five-equation or a
    viscous material, a NaN step and a negative step count are refused."""
    import paper_2402_05193_gb300 as jxf
    P = jxf.JXF_BC_PERIODIC
    grid = jxf.ls_grid(3, [8, 8, 8], 0.1, [(P, P)] * 3)
    assert jxf.lib().jxf_ls_step_work(ctypes.byref(grid)) > 0
    bad = jxf.ls_grid(3, [8, 8, 8], 0.1, [(P, P)] * 3)
    bad.hi[2] = bad.lo[2] + 1.0
    assert jxf.lib().jxf_ls_step_work(ctypes.byref(bad)) == -1
    # 32-bit cell indices: 2^31 cells or more are refused, 2-cell axes too
    huge = jxf.ls_grid(3, [1300, 1300, 1300], 1e-3, [(P, P)] * 3)
    assert jxf.lib().jxf_ls_step_work(ctypes.byref(huge)) == -1
    thin = jxf.ls_grid(2, [8, 2], 0.1, [(P, P)] * 2)
    assert jxf.lib().jxf_ls_step_work(ctypes.byref(thin)) == -1
    big = jxf.ls_grid(3, [1200, 1200, 1200], 1e-3, [(P, P)] * 3)  # 1.73e9 cells: accepted
    assert jxf.lib().jxf_ls_step_work(ctypes.byref(big)) > 1200 ** 3

    def eos(g, pi, model=jxf.JXF_SPM):
        e = jxf.jxf_eos()
        e.model = model
        e.gamma[0] = e.gamma[1] = g
        e.pinf[0] = e.pinf[1] = pi
        return e

    sch = jxf.jxf_scheme()
    sch.recon, sch.precision, sch.weno_eps = jxf.JXF_WENO5JS_CHAR, jxf.JXF_FP64, 1e-6
    visc = jxf.jxf_scheme()
    visc.recon, visc.precision, visc.viscous = jxf.JXF_WENO5JS_CHAR, jxf.JXF_FP64, 1
    e1, e2 = eos(1.4, 0.0), eos(1.67, 0.0)
    ev1, ev2 = eos(1.4, 0.0), eos(1.67, 0.0)
    for e in (ev1, ev2):
        e.mu, e.Pr, e.R = 1e-3, 0.72, 287.0
    buf = (ctypes.c_double * 8)()  # never touched: every call below returns before any work
    p = ctypes.cast(buf, ctypes.c_void_p)
    cases = [(grid, eos(1.4, 0.0, jxf.JXF_DIM), e2, sch, 1e-3, 1, jxf.JXF_ERR_UNSUPPORTED),
             (grid, ev1, ev2, visc, 1e-3, 1, jxf.JXF_ERR_UNSUPPORTED),
             (grid, e1, e2, sch, float("nan"), 1, jxf.JXF_ERR_ARG),
             (grid, e1, e2, sch, 1e-3, -1, jxf.JXF_ERR_ARG),
             (bad, e1, e2, sch, 1e-3, 1, jxf.JXF_ERR_ARG),
             (grid, eos(0.9, 0.0), e2, sch, 1e-3, 1, jxf.JXF_ERR_ARG)]
    for g_, a, b, s_, dt, nst, code in cases:
        rc = jxf.lib().jxf_ls_step(ctypes.byref(g_), ctypes.byref(a), ctypes.byref(b), ctypes.byref(s_), dt, nst,
                                   0.6, p, p, p, p, p, p, p, None)
        assert rc == code, (dt, nst, rc)
    rc = jxf.lib().jxf_ls_init(ctypes.byref(grid), ctypes.byref(eos(1.4, 0.0, jxf.JXF_DIM)), ctypes.byref(e2),
                               ctypes.byref(sch), p, p, p, p, p, p, p, None)
    assert rc == jxf.JXF_ERR_UNSUPPORTED
