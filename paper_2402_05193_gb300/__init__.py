"""GB300-native (sm_103a) compressible-flow RHS / TVD-RK3 library.

Python binding of the C interface declared in ``include/jxf.h``: the
``jxf_*`` functions below carry the C names and only marshal arguments; every
step of the computation runs in the CUDA kernels of ``_build/libjxf.so``.
There is no CPU fallback: if the library is missing or cannot be loaded, every
call raises.

``Solver`` wraps a handle for the common case of torch tensors on the GPU (or
host numpy arrays / tensors, which the library copies itself).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# JXF_LIB selects another build of the same library (tuning variants)
LIB_PATH = os.environ.get("JXF_LIB", os.path.join(_HERE, "_build", "libjxf.so"))

JXF_OK, JXF_ERR_ARG, JXF_ERR_CUDA, JXF_ERR_OOM, JXF_ERR_NONPHYSICAL, JXF_ERR_TIMEOUT, \
    JXF_ERR_UNSUPPORTED, JXF_ERR_BOUNDS = range(8)
JXF_BC_PERIODIC, JXF_BC_ZEROGRAD, JXF_BC_SYMMETRY, JXF_BC_NEIGHBOR = 0, 1, 2, 3
JXF_PHASE_STAGE, JXF_PHASE_AUX, JXF_PHASE_REDUCE, JXF_PHASE_FINISH = 0, 1, 2, 3
JXF_HALO_STATE, JXF_HALO_AUX = 0, 1
JXF_RECORD_LEN = 10
JXF_SPM, JXF_DIM = 0, 1
JXF_WENO5JS_COMP, JXF_WENO5JS_CHAR, JXF_WENO5Z_COMP, JXF_WENO5Z_CHAR = 0, 1, 2, 3
JXF_TENO6A_COMP, JXF_TENO6A_CHAR = 4, 5
JXF_FP64, JXF_MIXED32 = 0, 1

_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NONPHYSICAL",
           5: "ERR_TIMEOUT", 6: "ERR_UNSUPPORTED", 7: "ERR_BOUNDS"}


class JxfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class jxf_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("bc", (ctypes.c_int * 2) * 3)]


class jxf_eos(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("gamma", ctypes.c_double * 2),
                ("pinf", ctypes.c_double * 2), ("mu", ctypes.c_double), ("Pr", ctypes.c_double),
                ("R", ctypes.c_double)]


class jxf_block(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int * 3), ("n", ctypes.c_int * 3), ("nbr", (ctypes.c_int * 2) * 3)]


class jxf_scheme(ctypes.Structure):
    _fields_ = [("recon", ctypes.c_int), ("viscous", ctypes.c_int), ("limiter", ctypes.c_int),
                ("precision", ctypes.c_int), ("cfl", ctypes.c_double),
                ("fixed_dt", ctypes.c_double), ("t_end", ctypes.c_double),
                ("eps_rho", ctypes.c_double), ("eps_rhoc2", ctypes.c_double),
                ("eps_alpha", ctypes.c_double), ("weno_eps", ctypes.c_double),
                ("thinc", ctypes.c_int), ("visc_order", ctypes.c_int)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libjxf.so (built by ``paper_2402_05193_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libjxf.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, H = ctypes.c_void_p, ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        L.jxf_create.argtypes = [ctypes.POINTER(jxf_grid), ctypes.POINTER(jxf_eos),
                                 ctypes.POINTER(jxf_scheme), ctypes.POINTER(H)]
        L.jxf_destroy.argtypes = [H]
        L.jxf_nvar.argtypes = [H]
        L.jxf_nvar.restype = ctypes.c_int
        L.jxf_ncell.argtypes = [H]
        L.jxf_ncell.restype = ctypes.c_longlong
        L.jxf_set_state.argtypes = [H, vp, vp]
        L.jxf_set_primitive.argtypes = [H, vp, vp]
        L.jxf_get_state.argtypes = [H, vp, vp]
        L.jxf_get_primitive.argtypes = [H, vp, vp]
        L.jxf_set_time.argtypes = [H, ctypes.c_double, vp]
        L.jxf_rhs.argtypes = [H, vp, vp, ctypes.c_double, vp]
        L.jxf_step.argtypes = [H, ctypes.c_int, dp, vp]
        L.jxf_stats.argtypes = [H, dp, dp, ctypes.POINTER(ctypes.c_longlong)]
        L.jxf_step_profiled.argtypes = [H, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_int), vp]
        L.jxf_rhs_vjp.argtypes = [H, vp, vp, vp, ctypes.c_double, vp]
        L.jxf_step_vjp.argtypes = [H, vp, ctypes.c_double, vp, vp, vp]
        L.jxf_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(jxf_grid), ctypes.POINTER(jxf_eos),
                                       ctypes.POINTER(jxf_scheme), ctypes.POINTER(H)]
        L.jxf_batch_destroy.argtypes = [H]
        L.jxf_batch_nsim.argtypes = [H]
        L.jxf_batch_nsim.restype = ctypes.c_int
        L.jxf_batch_set_primitive.argtypes = [H, ctypes.c_int, vp, vp]
        L.jxf_batch_set_state.argtypes = [H, ctypes.c_int, vp, vp]
        L.jxf_batch_set_time.argtypes = [H, ctypes.c_int, ctypes.c_double, vp]
        L.jxf_batch_get_state.argtypes = [H, ctypes.c_int, vp, vp]
        L.jxf_batch_set_tiling.argtypes = [H, ctypes.c_int, ctypes.c_int]
        L.jxf_batch_step.argtypes = [H, ctypes.c_int, vp]
        L.jxf_batch_stats.argtypes = [H, ctypes.c_int, dp, dp, dp, ctypes.POINTER(ctypes.c_longlong)]
        L.jxf_batch_last_error.argtypes = [H]
        L.jxf_batch_last_error.restype = ctypes.c_char_p
        for name in ("jxf_batch_create", "jxf_batch_destroy", "jxf_batch_set_primitive",
                     "jxf_batch_set_state", "jxf_batch_set_time", "jxf_batch_get_state",
                     "jxf_batch_set_tiling", "jxf_batch_step", "jxf_batch_stats"):
            getattr(L, name).restype = ctypes.c_int
        L.jxf_create_block.argtypes = [ctypes.POINTER(jxf_grid), ctypes.POINTER(jxf_eos),
                                       ctypes.POINTER(jxf_scheme), ctypes.POINTER(jxf_block),
                                       ctypes.POINTER(H)]
        L.jxf_block_phase.argtypes = [H, ctypes.c_int, ctypes.c_int, vp]
        L.jxf_block_halo_count.argtypes = [H, ctypes.c_int]
        L.jxf_block_halo_count.restype = ctypes.c_int
        L.jxf_block_halo.argtypes = [H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int)]
        L.jxf_block_exchange.argtypes = [H, H, ctypes.c_int, vp]
        L.jxf_block_record.argtypes = [H, ctypes.POINTER(vp)]
        L.jxf_block_allreduce.argtypes = [ctypes.POINTER(H), ctypes.c_int, vp]
        for name in ("jxf_create_block", "jxf_block_phase", "jxf_block_halo", "jxf_block_exchange",
                     "jxf_block_record", "jxf_block_allreduce"):
            getattr(L, name).restype = ctypes.c_int
        G = ctypes.POINTER(jxf_grid)
        L.jxf_ls_nface.argtypes = [G]
        L.jxf_ls_nface.restype = ctypes.c_longlong
        L.jxf_ls_geometry.argtypes = [G, vp, vp, vp, vp, vp, vp]
        L.jxf_ls_rhs.argtypes = [G, vp, vp, vp, vp]
        L.jxf_ls_advect.argtypes = [G, vp, vp, ctypes.c_double, ctypes.c_int, vp, vp]
        L.jxf_ls_reinit_rhs.argtypes = [G, vp, vp, ctypes.c_double, vp, vp]
        L.jxf_ls_reinit.argtypes = [G, vp, ctypes.c_int, ctypes.c_double, vp, vp]
        L.jxf_ls_interface.argtypes = [G, vp, vp, dp, dp, vp, vp, vp, vp, vp, vp]
        L.jxf_ls_extend.argtypes = [G, vp, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
        L.jxf_ls_cut_rhs.argtypes = [G, ctypes.POINTER(jxf_eos), ctypes.POINTER(jxf_scheme), vp, vp, vp, vp,
                                     ctypes.c_int, vp, vp, vp, vp, vp]
        L.jxf_ls_mix.argtypes = [G, ctypes.c_int, vp, vp, vp, ctypes.c_double, vp, vp, vp]
        E, S = ctypes.POINTER(jxf_eos), ctypes.POINTER(jxf_scheme)
        L.jxf_ls_step_work.argtypes = [G]
        L.jxf_ls_step_work.restype = ctypes.c_longlong
        L.jxf_ls_init.argtypes = [G, E, E, S, vp, vp, vp, vp, vp, vp, vp, vp]
        L.jxf_ls_step.argtypes = [G, E, E, S, ctypes.c_double, ctypes.c_int, ctypes.c_double, vp, vp, vp, vp, vp,
                                  vp, vp, vp]
        for name in ("jxf_ls_geometry", "jxf_ls_rhs", "jxf_ls_advect", "jxf_ls_reinit_rhs", "jxf_ls_reinit",
                     "jxf_ls_interface", "jxf_ls_extend", "jxf_ls_cut_rhs", "jxf_ls_mix", "jxf_ls_init",
                     "jxf_ls_step"):
            getattr(L, name).restype = ctypes.c_int
        L.jxf_last_error.argtypes = [H]
        L.jxf_last_error.restype = ctypes.c_char_p
        for name in ("jxf_create", "jxf_destroy", "jxf_set_state", "jxf_set_primitive",
                     "jxf_get_state", "jxf_get_primitive", "jxf_set_time", "jxf_rhs", "jxf_step",
                     "jxf_stats", "jxf_step_profiled", "jxf_rhs_vjp", "jxf_step_vjp"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(h, status):
    if status != JXF_OK:
        msg = lib().jxf_last_error(h)
        raise JxfError(status, msg.decode() if msg else "")


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return ctypes.c_void_p(a.ctypes.data)
    assert a.is_contiguous()
    return ctypes.c_void_p(a.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream) if torch.cuda.is_available() \
            else ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ------------------------------------------------------- C-named functions --
def jxf_create(grid: jxf_grid, eos: jxf_eos, scheme: jxf_scheme):
    h = ctypes.c_void_p()
    _check(None, lib().jxf_create(ctypes.byref(grid), ctypes.byref(eos), ctypes.byref(scheme),
                                  ctypes.byref(h)))
    return h


def jxf_destroy(h):
    _check(h, lib().jxf_destroy(h))


def jxf_nvar(h) -> int:
    return lib().jxf_nvar(h)


def jxf_ncell(h) -> int:
    return lib().jxf_ncell(h)


def jxf_set_state(h, U, stream=None):
    _check(h, lib().jxf_set_state(h, _ptr(U), _stream(stream)))


def jxf_set_primitive(h, W, stream=None):
    _check(h, lib().jxf_set_primitive(h, _ptr(W), _stream(stream)))


def jxf_get_state(h, U, stream=None):
    _check(h, lib().jxf_get_state(h, _ptr(U), _stream(stream)))


def jxf_get_primitive(h, W, stream=None):
    _check(h, lib().jxf_get_primitive(h, _ptr(W), _stream(stream)))


def jxf_set_time(h, t: float, stream=None):
    _check(h, lib().jxf_set_time(h, float(t), _stream(stream)))


def jxf_rhs(h, U, dU, dt: float = 0.0, stream=None):
    _check(h, lib().jxf_rhs(h, _ptr(U), _ptr(dU), float(dt), _stream(stream)))


def jxf_step(h, n: int, sync: bool = True, stream=None):
    """n TVD-RK3 steps; returns the simulation time if sync, else None."""
    t = ctypes.c_double(0.0)
    _check(h, lib().jxf_step(h, int(n), ctypes.byref(t) if sync else None, _stream(stream)))
    return t.value if sync else None


def jxf_rhs_vjp(h, U, R_bar, U_bar, dt: float = 0.0, stream=None):
    _check(h, lib().jxf_rhs_vjp(h, _ptr(U), _ptr(R_bar), _ptr(U_bar), float(dt), _stream(stream)))


def jxf_step_vjp(h, U_n, dt: float, U_bar_np1, U_bar_n, stream=None):
    _check(h, lib().jxf_step_vjp(h, _ptr(U_n), float(dt), _ptr(U_bar_np1), _ptr(U_bar_n),
                                 _stream(stream)))


KERNEL_KINDS = ("flux_x", "flux_y", "flux_z", "update", "finalize")


def jxf_step_profiled(h, n: int, stream=None):
    """n steps with per-kernel event timing: {kind: (ms total, launches)}."""
    ms = (ctypes.c_float * 5)()
    cnt = (ctypes.c_int * 5)()
    _check(h, lib().jxf_step_profiled(h, int(n), ms, cnt, _stream(stream)))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def jxf_fail_allocation_after(k: int):
    """Host-side fault injection: the k-th following device allocation of a
    handle fails as if out of memory (k < 0 disarms)."""
    L = lib()
    L.jxf_fail_allocation_after.argtypes = [ctypes.c_int]
    L.jxf_fail_allocation_after.restype = None
    L.jxf_fail_allocation_after(int(k))


def jxf_peak_probe(precision: int) -> float:
    """Measured FMA throughput (TFLOP/s) of the plain ALUs in FP64 or FP32."""
    L = lib()
    L.jxf_peak_probe.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.jxf_peak_probe.restype = ctypes.c_int
    out = ctypes.c_double(0.0)
    _check(None, L.jxf_peak_probe(int(precision), ctypes.byref(out)))
    return out.value


def jxf_stats(h):
    nv = jxf_nvar(h)
    sums = (ctypes.c_double * nv)()
    dl = ctypes.c_double(0.0)
    lim = (ctypes.c_longlong * 2)()
    _check(h, lib().jxf_stats(h, sums, ctypes.byref(dl), lim))
    return np.array(sums[:]), dl.value, (lim[0], lim[1])


def jxf_create_block(grid: jxf_grid, eos: jxf_eos, scheme: jxf_scheme, block: jxf_block):
    h = ctypes.c_void_p()
    _check(None, lib().jxf_create_block(ctypes.byref(grid), ctypes.byref(eos), ctypes.byref(scheme),
                                        ctypes.byref(block), ctypes.byref(h)))
    return h


def jxf_block_phase(h, phase: int, arg: int = 0, stream=None):
    _check(h, lib().jxf_block_phase(h, int(phase), int(arg), _stream(stream)))


def jxf_block_halo_count(h, kind: int) -> int:
    n = lib().jxf_block_halo_count(h, int(kind))
    if n < 0:
        raise JxfError(JXF_ERR_ARG, "jxf_block_halo_count: not a block handle or bad kind")
    return n


def jxf_block_halo(h, kind: int, index: int, side: int, recv: int):
    """(device pointer, pitch bytes, width bytes, rows) of one halo region."""
    ptr, pitch, width, height = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int()
    _check(h, lib().jxf_block_halo(h, int(kind), int(index), int(side), int(recv), ctypes.byref(ptr),
                                   ctypes.byref(pitch), ctypes.byref(width), ctypes.byref(height)))
    return ptr.value, pitch.value, width.value, height.value


def jxf_block_exchange(lo, hi, kind: int, stream=None):
    _check(lo, lib().jxf_block_exchange(lo, hi, int(kind), _stream(stream)))


def jxf_block_record(h) -> int:
    ptr = ctypes.c_void_p()
    _check(h, lib().jxf_block_record(h, ctypes.byref(ptr)))
    return ptr.value


def jxf_block_allreduce(blocks, stream=None):
    arr = (ctypes.c_void_p * len(blocks))(*[b.value for b in blocks])
    _check(blocks[0], lib().jxf_block_allreduce(arr, len(blocks), _stream(stream)))


def jxf_rhs_static(grid: jxf_grid, eos: jxf_eos, scheme: jxf_scheme, U, dU, dt: float = 0.0,
                   stream=None):
    """dU = R(U) through the allocation-free entry point (device tensors of
    the current device; see include/jxf.h)."""
    L = lib()
    f = L.jxf_rhs_static
    f.argtypes = [ctypes.POINTER(jxf_grid), ctypes.POINTER(jxf_eos), ctypes.POINTER(jxf_scheme),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_char_p, ctypes.c_size_t]
    f.restype = ctypes.c_int
    msg = ctypes.create_string_buffer(256)
    st = f(ctypes.byref(grid), ctypes.byref(eos), ctypes.byref(scheme), _ptr(U), _ptr(dU),
           float(dt), _stream(stream), msg, 256)
    if st != JXF_OK:
        raise JxfError(st, msg.value.decode())


# ---------------------------------------------------------------- Solver ----
_BC = {"periodic": JXF_BC_PERIODIC, "zerograd": JXF_BC_ZEROGRAD, "symmetry": JXF_BC_SYMMETRY}


def structs_from_case(case: dict, precision: str = "fp64", **over):
    """C structs for a workload dict (see ``workloads``).  Scheme keys:
    ``recon`` ("comp" | "char"), ``weno`` ("js" | "z" | "teno6a"), ``viscous``,
    ``visc_order`` (2 | 4 | 6), ``limiter``, ``thinc`` (five-equation model),
    ``cfl``, ``fixed_dt``, ``t_end``, optional ``eps`` and ``weno_eps``;
    ``over`` replaces keys."""
    c = dict(case)
    c.update(over)
    g = jxf_grid()
    g.ndim = c["ndim"]
    for e in range(3):
        if e < c["ndim"]:
            g.n[e] = c["n"][e]
            g.lo[e] = c["lo"][e] if "lo" in c else 0.0
            g.hi[e] = g.lo[e] + c["n"][e] * c["dx"][e]
            g.bc[e][0], g.bc[e][1] = _BC[c["bc"][e][0]], _BC[c["bc"][e][1]]
        else:
            g.n[e], g.lo[e], g.hi[e] = 1, 0.0, 1.0
            g.bc[e][0] = g.bc[e][1] = JXF_BC_ZEROGRAD
    eo = jxf_eos()
    eo.model = JXF_DIM if c["model"] == "dim" else JXF_SPM
    eo.gamma[0], eo.gamma[1] = c["gamma"]
    eo.pinf[0], eo.pinf[1] = c["pinf"]
    eo.mu, eo.Pr, eo.R = c["mu"], c["Pr"], c["R"]
    s = jxf_scheme()
    s.recon = (JXF_WENO5JS_CHAR if c["recon"] == "char" else JXF_WENO5JS_COMP) + \
        {"js": 0, "z": 2, "teno6a": 4}[c.get("weno", "js")]
    s.viscous = int(bool(c["viscous"]))
    s.limiter = int(bool(c["limiter"]))
    s.precision = JXF_FP64 if precision == "fp64" else JXF_MIXED32
    s.cfl, s.fixed_dt, s.t_end = c["cfl"], c["fixed_dt"], c["t_end"]
    eps = c.get("eps")
    if eps is not None:
        s.eps_rho, s.eps_rhoc2, s.eps_alpha = eps
    s.weno_eps = c.get("weno_eps", 0.0)
    s.thinc = int(bool(c.get("thinc", False)))
    s.visc_order = int(c.get("visc_order", 4))
    return g, eo, s


def _bcheck(b, status):
    if status != JXF_OK:
        msg = lib().jxf_batch_last_error(b)
        raise JxfError(status, msg.decode() if msg else "")


def jxf_batch_create(grids, eos: jxf_eos, scheme: jxf_scheme):
    arr = (jxf_grid * len(grids))(*grids)
    b = ctypes.c_void_p()
    _bcheck(None, lib().jxf_batch_create(len(grids), arr, ctypes.byref(eos), ctypes.byref(scheme),
                                         ctypes.byref(b)))
    return b


def jxf_batch_destroy(b):
    _bcheck(b, lib().jxf_batch_destroy(b))


def jxf_batch_set_primitive(b, sim: int, W, stream=None):
    _bcheck(b, lib().jxf_batch_set_primitive(b, sim, _ptr(W), _stream(stream)))


def jxf_batch_set_state(b, sim: int, U, stream=None):
    _bcheck(b, lib().jxf_batch_set_state(b, sim, _ptr(U), _stream(stream)))


def jxf_batch_get_state(b, sim: int, U, stream=None):
    _bcheck(b, lib().jxf_batch_get_state(b, sim, _ptr(U), _stream(stream)))


def jxf_batch_set_tiling(b, tile_faces: int, blocks_per_sm: int):
    _bcheck(b, lib().jxf_batch_set_tiling(b, int(tile_faces), int(blocks_per_sm)))


def jxf_batch_step(b, n: int, stream=None):
    _bcheck(b, lib().jxf_batch_step(b, int(n), _stream(stream)))


def jxf_batch_stats(b, sim: int, nv: int):
    t, dl = ctypes.c_double(0.0), ctypes.c_double(0.0)
    sums = (ctypes.c_double * nv)()
    lim = (ctypes.c_longlong * 2)()
    _bcheck(b, lib().jxf_batch_stats(b, sim, ctypes.byref(t), sums, ctypes.byref(dl), lim))
    return t.value, np.array(sums[:]), dl.value, (lim[0], lim[1])


class Batch:
    """Many independent simulations (workload dicts of one model, scheme and
    dimension, uneven sizes) advanced together on the current CUDA device."""

    def __init__(self, cases, precision: str = "fp64"):
        structs = [structs_from_case(c, precision) for c in cases]
        self.cases = cases
        self.precision = precision
        self.b = jxf_batch_create([g for g, _, _ in structs], structs[0][1], structs[0][2])
        self.nv = cases[0]["W"].shape[0]
        self.shapes = [c["W"].shape for c in cases]

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def close(self):
        if getattr(self, "b", None):
            jxf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_primitives(self, stream=None):
        for k, c in enumerate(self.cases):
            jxf_batch_set_primitive(self.b, k, np.ascontiguousarray(c["W"], dtype=np.float64), stream)

    def state(self, sim: int, stream=None):
        import torch
        out = torch.empty(self.shapes[sim], dtype=self.dtype, device="cuda")
        jxf_batch_get_state(self.b, sim, out, stream)
        return out

    def step(self, n: int, stream=None):
        jxf_batch_step(self.b, n, stream)

    def stats(self, sim: int):
        return jxf_batch_stats(self.b, sim, self.nv)

    def set_tiling(self, tile_faces: int, blocks_per_sm: int):
        jxf_batch_set_tiling(self.b, tile_faces, blocks_per_sm)


class Solver:
    """One simulation on the current CUDA device."""

    def __init__(self, case: dict, precision: str = "fp64", **over):
        self.case = case
        self.precision = precision
        self.h = jxf_create(*structs_from_case(case, precision, **over))
        self.nv = jxf_nvar(self.h)
        self.ncell = jxf_ncell(self.h)
        n = list(case["n"]) + [1] * (3 - case["ndim"])
        self.shape = (self.nv, n[2], n[1], n[0])

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def close(self):
        if getattr(self, "h", None):
            jxf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_primitive(self, W, stream=None):
        """W: float64 primitive field (host numpy / tensor or device tensor)."""
        if isinstance(W, np.ndarray):
            W = np.ascontiguousarray(W, dtype=np.float64)
        jxf_set_primitive(self.h, W, stream)

    def set_state(self, U, stream=None):
        jxf_set_state(self.h, U, stream)

    def state(self, stream=None):
        import torch
        out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        jxf_get_state(self.h, out, stream)
        return out

    def primitive(self, stream=None):
        import torch
        out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        jxf_get_primitive(self.h, out, stream)
        return out

    def rhs(self, U, dt: float = 0.0, stream=None):
        import torch
        dU = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        jxf_rhs(self.h, U, dU, dt, stream)
        return dU

    def step(self, n: int, sync: bool = True, stream=None):
        return jxf_step(self.h, n, sync, stream)

    def set_time(self, t: float, stream=None):
        jxf_set_time(self.h, t, stream)

    def stats(self):
        return jxf_stats(self.h)

    def step_profiled(self, n: int, stream=None):
        return jxf_step_profiled(self.h, n, stream)

    def rhs_vjp(self, U, R_bar, stream=None):
        """(dR/dU)^T R_bar at U (device tensors)."""
        import torch
        out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        jxf_rhs_vjp(self.h, U, R_bar.contiguous(), out, 0.0, stream)
        return out

    def step_vjp(self, U_n, dt: float, U_bar_np1, stream=None):
        """(dU^{n+1}/dU^n)^T U_bar_np1 for one RK3 step of size dt from U_n."""
        import torch
        out = torch.empty(self.shape, dtype=self.dtype, device="cuda")
        jxf_step_vjp(self.h, U_n, dt, U_bar_np1.contiguous(), out, stream)
        return out


# ------------------------------------------------------------------ level set --
# The level-set model's data-parallel parts (§3.5, App. D) on device arrays
# (FP64 torch tensors of the cells, x fastest): the C calls of the same names.
def ls_grid(ndim: int, n, h: float, bc) -> jxf_grid:
    """A grid of cubic cells of size h for the level-set calls."""
    g = jxf_grid()
    g.ndim = ndim
    for e in range(3):
        g.n[e] = int(n[e]) if e < ndim else 1
        g.lo[e] = 0.0
        g.hi[e] = h * g.n[e] if e < ndim else 1.0
        b = bc[e] if e < len(bc) else (JXF_BC_ZEROGRAD, JXF_BC_ZEROGRAD)
        g.bc[e][0], g.bc[e][1] = b
    return g


def _ls_status(status):
    if status != JXF_OK:
        msg = {JXF_ERR_ARG: "invalid grid or argument", JXF_ERR_UNSUPPORTED: "unsupported model or scheme"}
        raise JxfError(status, "jxf_ls: " + msg.get(status, "CUDA failure"))


def jxf_ls_nface(grid: jxf_grid) -> int:
    return int(lib().jxf_ls_nface(ctypes.byref(grid)))


def jxf_ls_geometry(grid: jxf_grid, phi, apert, alpha, dgamma, normal, stream=None):
    _ls_status(lib().jxf_ls_geometry(ctypes.byref(grid), _ptr(phi), _ptr(apert), _ptr(alpha), _ptr(dgamma),
                                     _ptr(normal), _stream(stream)))


def jxf_ls_rhs(grid: jxf_grid, phi, vel, rhs, stream=None):
    _ls_status(lib().jxf_ls_rhs(ctypes.byref(grid), _ptr(phi), _ptr(vel), _ptr(rhs), _stream(stream)))


def jxf_ls_advect(grid: jxf_grid, phi, vel, dt: float, nsteps: int, scratch, stream=None):
    _ls_status(lib().jxf_ls_advect(ctypes.byref(grid), _ptr(phi), _ptr(vel), float(dt), int(nsteps),
                                   _ptr(scratch), _stream(stream)))


def jxf_ls_reinit_rhs(grid: jxf_grid, phi, phi0, threshold: float, rhs, stream=None):
    _ls_status(lib().jxf_ls_reinit_rhs(ctypes.byref(grid), _ptr(phi), _ptr(phi0), float(threshold), _ptr(rhs),
                                       _stream(stream)))


def jxf_ls_reinit(grid: jxf_grid, phi, steps: int, threshold: float, scratch, stream=None):
    _ls_status(lib().jxf_ls_reinit(ctypes.byref(grid), _ptr(phi), int(steps), float(threshold), _ptr(scratch),
                                   _stream(stream)))


def jxf_ls_interface(grid: jxf_grid, W1, W2, gamma, pinf, alpha, dgamma, normal, ug, pg, stream=None):
    ga = (ctypes.c_double * 2)(*gamma)
    pa = (ctypes.c_double * 2)(*pinf)
    _ls_status(lib().jxf_ls_interface(ctypes.byref(grid), _ptr(W1), _ptr(W2), ga, pa, _ptr(alpha), _ptr(dgamma),
                                      _ptr(normal), _ptr(ug), _ptr(pg), _stream(stream)))


def jxf_ls_extend(grid: jxf_grid, phi, alpha, dgamma, normal, q, nq: int, mode: int, steps: int, scratch,
                  stream=None):
    _ls_status(lib().jxf_ls_extend(ctypes.byref(grid), _ptr(phi), _ptr(alpha), _ptr(dgamma), _ptr(normal), _ptr(q),
                                   int(nq), int(mode), int(steps), _ptr(scratch), _stream(stream)))


def jxf_ls_cut_rhs(grid: jxf_grid, eos: jxf_eos, scheme: jxf_scheme, apert, dgamma, normal, W, phase: int, ug, pg,
                   dU, scratch, stream=None):
    _ls_status(lib().jxf_ls_cut_rhs(ctypes.byref(grid), ctypes.byref(eos), ctypes.byref(scheme), _ptr(apert),
                                    _ptr(dgamma), _ptr(normal), _ptr(W), int(phase), _ptr(ug), _ptr(pg), _ptr(dU),
                                    _ptr(scratch), _stream(stream)))


def jxf_ls_mix(grid: jxf_grid, nv: int, a0, a1, np_, amix: float, aU, scratch, stream=None):
    _ls_status(lib().jxf_ls_mix(ctypes.byref(grid), int(nv), _ptr(a0), _ptr(a1), _ptr(np_), float(amix), _ptr(aU),
                                _ptr(scratch), _stream(stream)))



def jxf_ls_step_work(grid: jxf_grid) -> int:
    """Doubles of the work buffer jxf_ls_init / jxf_ls_step take."""
    n = int(lib().jxf_ls_step_work(ctypes.byref(grid)))
    if n < 0:
        raise ValueError("jxf_ls_step_work: invalid level-set grid")
    return n


def jxf_ls_init(grid: jxf_grid, eos1: jxf_eos, eos2: jxf_eos, scheme: jxf_scheme, phi, W1, W2, aU1, aU2, qg, work,
                stream=None):
    _ls_status(lib().jxf_ls_init(ctypes.byref(grid), ctypes.byref(eos1), ctypes.byref(eos2), ctypes.byref(scheme),
                                 _ptr(phi), _ptr(W1), _ptr(W2), _ptr(aU1), _ptr(aU2), _ptr(qg), _ptr(work),
                                 _stream(stream)))


def jxf_ls_step(grid: jxf_grid, eos1: jxf_eos, eos2: jxf_eos, scheme: jxf_scheme, dt: float, nsteps: int,
                amix: float, phi, aU1, aU2, W1, W2, qg, work, stream=None):
    _ls_status(lib().jxf_ls_step(ctypes.byref(grid), ctypes.byref(eos1), ctypes.byref(eos2), ctypes.byref(scheme),
                                 float(dt), int(nsteps), float(amix), _ptr(phi), _ptr(aU1), _ptr(aU2), _ptr(W1),
                                 _ptr(W2), _ptr(qg), _ptr(work), _stream(stream)))

_RECON = {"js_comp": JXF_WENO5JS_COMP, "js_char": JXF_WENO5JS_CHAR, "z_comp": JXF_WENO5Z_COMP,
          "z_char": JXF_WENO5Z_CHAR, "teno6a_comp": JXF_TENO6A_COMP, "teno6a_char": JXF_TENO6A_CHAR}


class LevelSet:
    """A two-phase level-set simulation on the current CUDA device (FP64):
    phase 1 (phi > 0) and phase 2 with their stiffened gases mat1, mat2 =
    (gamma, p_inf), on a grid of cubic cells of size h, one reconstruction
    ("js_char", "z_char", "teno6a_char", ... see _RECON).  The state lives in
    device tensors: phi, W1, W2 (rho, u_d, p of each phase, extended into its
    ghost cells), aU1, aU2 (the volume-weighted conservative states) and qg
    (u_Gamma n component by component, then p_Gamma); every step runs
    through jxf_ls_step."""

    def __init__(self, ndim: int, n, h: float, bc, mat1, mat2, recon: str = "js_char", amix: float = 0.6):
        import torch
        self.ndim, self.h, self.amix = ndim, float(h), float(amix)
        self.grid = ls_grid(ndim, n, h, bc)
        self.shape = tuple(int(n[e]) for e in reversed(range(ndim)))
        self.eos = []
        for g, pi in (mat1, mat2):
            e = jxf_eos()
            e.model = JXF_SPM
            e.gamma[0] = e.gamma[1] = float(g)
            e.pinf[0] = e.pinf[1] = float(pi)
            self.eos.append(e)
        self.scheme = jxf_scheme()
        self.scheme.recon, self.scheme.precision, self.scheme.weno_eps = _RECON[recon], JXF_FP64, 1e-6
        z = lambda *lead: torch.zeros(lead + self.shape, dtype=torch.float64, device="cuda")  # noqa: E731
        self.phi, self.W1, self.W2 = z(), z(ndim + 2), z(ndim + 2)
        self.aU1, self.aU2, self.qg = z(ndim + 2), z(ndim + 2), z(ndim + 1)
        self.work = torch.zeros(jxf_ls_step_work(self.grid), dtype=torch.float64, device="cuda")

    def set_state(self, phi, W1, W2, stream=None):
        """The level set and both phases' primitives in every cell (host or
        device arrays); forms the volume-weighted states and the interface
        quantities."""
        import torch
        for dst, src in ((self.phi, phi), (self.W1, W1), (self.W2, W2)):
            dst.copy_(torch.as_tensor(np.ascontiguousarray(src) if isinstance(src, np.ndarray) else src))
        jxf_ls_init(self.grid, self.eos[0], self.eos[1], self.scheme, self.phi, self.W1, self.W2, self.aU1,
                    self.aU2, self.qg, self.work, stream)

    def step(self, dt: float, n: int = 1, stream=None):
        jxf_ls_step(self.grid, self.eos[0], self.eos[1], self.scheme, dt, n, self.amix, self.phi, self.aU1,
                    self.aU2, self.W1, self.W2, self.qg, self.work, stream)

    def geometry(self, stream=None):
        """(apertures, alpha, dGamma, normal) of the current level set."""
        import torch
        ap = torch.zeros(jxf_ls_nface(self.grid), dtype=torch.float64, device="cuda")
        al = torch.zeros(self.shape, dtype=torch.float64, device="cuda")
        dg = torch.zeros_like(al)
        nr = torch.zeros((self.ndim,) + self.shape, dtype=torch.float64, device="cuda")
        jxf_ls_geometry(self.grid, self.phi, ap, al, dg, nr, stream)
        return ap, al, dg, nr
