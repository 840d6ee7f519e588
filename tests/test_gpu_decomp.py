"""One grid decomposed into blocks on one GPU (§4.2, §4.3, Alg. 1): blocks
of the grid split into slabs along its last active axis, each a handle of
its own, stepped phase by phase with the halo exchange between the blocks
and the reduction of their records, through the C interface.  The blocks
hold the same values, bit for bit, as one handle on the whole grid: the same
kernels do the same arithmetic on the same cells, the block sides only
change where a stencil finds its neighbours.  The time step (a maximum and a
minimum over all cells) and the limiter counts match exactly; the
conservation sums, reduced in another order, to round-off."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2402_05193_gb300 as jxf  # noqa: E402
from paper_2402_05193_gb300 import workloads as wl  # noqa: E402
from paper_2402_05193_gb300.decomp import SlabGrid  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _single(case, prec, steps):
    s = jxf.Solver(case, prec)
    s.set_primitive(case["W"])
    s.step(steps)
    U = s.state().cpu().numpy()
    sums, dt, lim = s.stats()
    s.close()
    return U, sums, dt, lim


def _blocks(case, prec, steps, nblocks):
    g = SlabGrid(case, prec, nblocks)
    g.set_primitive(case["W"])
    g.step(steps)
    U = g.state().cpu().numpy()
    sums, dt, lim = g.stats()
    g.close()
    return U, sums, dt, lim


CASES = {
    # the benchmark's scheme: characteristic WENO5-JS, 4th-order viscous, periodic
    "tgv32_2": (lambda: wl.tgv(32), 50, 2),
    "tgv32_4": (lambda: wl.tgv(32), 20, 4),
    # one block over the periodic axis: it exchanges with itself
    "tgv16_1": (lambda: wl.tgv(16), 20, 1),
    # TENO6-A with the 6th-order viscous stencils (three planes deep)
    "tgv32_teno6a_visc6_2": (lambda: dict(wl.tgv(32), weno="teno6a", visc_order=6), 20, 2),
    # five-equation model with both limiters, zero-gradient ends of the split axis
    "shock_bubble_2": (lambda: wl.shock_bubble(32, 16, 16), 30, 2),
    # THINC (the interface normal and smoothed volume fraction cross the sides)
    "shock_bubble_thinc_2": (lambda: dict(wl.shock_bubble(32, 16, 16, offset=(0.31, 0.17, 0.23)),
                                          thinc=True), 30, 2),
    # symmetry and zero-gradient sides of the grid on the split axis
    "sym_zerograd_2": (lambda: dict(wl.smooth_random(3, [12, 10, 16], "spm", seed=3, recon="comp"),
                                    bc=[("symmetry", "zerograd"), ("zerograd", "symmetry"),
                                        ("symmetry", "zerograd")]), 20, 2),
    # a 2-D grid split along y
    "kh64_2d_2": (lambda: wl.kelvin_helmholtz(64, steps=40), 40, 2),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_blocks_equal_the_single_grid_bit_for_bit(name, prec):
    make, steps, nblocks = CASES[name]
    case = make()
    U1, s1, dt1, lim1 = _single(case, prec, steps)
    Ub, sb, dtb, limb = _blocks(case, prec, steps, nblocks)
    scale = np.maximum(np.abs(s1), np.abs(U1).reshape(U1.shape[0], -1).sum(axis=1) * np.prod(case["dx"]))
    sums = np.abs(sb - s1) / np.where(scale > 0, scale, 1.0)
    diff = np.abs(Ub.astype(np.float64) - U1.astype(np.float64)).max()
    print("%s, %s, %d blocks, %d steps: max |U_blocks - U_grid| = %.3g, dt %.17g / %.17g, limited %s / %s, "
          "sums rel %s" % (name, prec, nblocks, steps, diff, dtb, dt1, limb, lim1, sums))
    assert np.array_equal(Ub, U1), diff
    assert dtb == dt1
    assert limb == lim1
    assert sums.max() < (1e-13 if prec == "fp64" else 1e-12)


def test_block_handles_reject_whole_grid_calls_and_bad_splits():
    case = wl.tgv(16)
    g = SlabGrid(case, "fp64", 2)
    with pytest.raises(jxf.JxfError) as ex:
        jxf.jxf_step(g.h[0], 1)
    assert ex.value.status == jxf.JXF_ERR_UNSUPPORTED
    with pytest.raises(jxf.JxfError):
        jxf.jxf_rhs(g.h[0], torch.zeros((5, 8, 16, 16), dtype=torch.float64, device="cuda"),
                    torch.zeros((5, 8, 16, 16), dtype=torch.float64, device="cuda"))
    g.close()
    g = SlabGrid(wl.shock_bubble(32, 16, 16), "fp64", 2)  # zero-gradient ends of the split axis
    with pytest.raises(jxf.JxfError):  # the upper block has no block above it
        jxf.jxf_block_exchange(g.h[1], g.h[0], jxf.JXF_HALO_STATE)
    g.close()
    gr, eo, sc = jxf.structs_from_case(case, "fp64")
    from paper_2402_05193_gb300.decomp import block_struct
    for lo, n, shared in (([0, 0, 0], [16, 16, 2], (True, True)),      # fewer than 3 planes
                          ([0, 0, 4], [16, 16, 8], (False, True)),     # inner side without a neighbour
                          ([0, 0, 0], [16, 8, 8], (True, True)),       # split along another axis
                          ([0, 0, 10], [16, 16, 8], (True, True))):    # beyond the grid
        with pytest.raises(jxf.JxfError) as ex:
            jxf.jxf_create_block(gr, eo, sc, block_struct(lo, n, shared, 3))
        assert ex.value.status == jxf.JXF_ERR_ARG


def test_dist_slab_on_one_rank_equals_the_single_grid():
    """The per-rank driver (halo regions as device tensors, the record
    reduced through torch.distributed) on a one-rank NCCL group: its block
    covers the periodic grid and exchanges with itself."""
    import os
    import socket

    import torch.distributed as dist
    from paper_2402_05193_gb300.decomp import DistSlab
    if dist.is_initialized():
        pytest.skip("a process group is already initialised")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        case = wl.tgv(16)
        for prec in ("fp64", "fp32"):
            U1, s1, dt1, _ = _single(case, prec, 20)
            d = DistSlab(case, prec)
            d.set_primitive(case["W"])
            d.step(20)
            Ud = d.state().cpu().numpy()
            sums, dt, _ = d.stats()
            d.close()
            print("DistSlab, one rank, %s: max diff %.3g, dt %.17g / %.17g"
                  % (prec, np.abs(Ud.astype(np.float64) - U1).max(), dt, dt1))
            assert np.array_equal(Ud, U1) and dt == dt1
    finally:
        dist.destroy_process_group()
