"""One grid decomposed into blocks: the homogeneous domain decomposition of
§4.2 with the halo update of §4.3 and the time-step reduction of Alg. 1.

The grid is split into equal slabs along its last active axis (z in 3-D), one
block per handle (``jxf_create_block``).  Each RK stage of a step is

    face sweeps + cell update          (jxf_block_phase STAGE s)
    halo exchange of the new state     (primitives, temperature, limiter
                                        state, THINC's smoothed fraction)
    auxiliary pass                     (velocity gradient / THINC normal)
    halo exchange of its result,

and after the third stage every block folds its reduction partials into a
record (max CFL rate, min density, admissibility, conservation sums) that is
reduced over all blocks before each block takes the next dt from it.  The
library's kernels do all the arithmetic; this module only moves halo planes
and records between blocks:

- ``SlabGrid``: all blocks in this process on the current device, moved
  with ``jxf_block_exchange`` / ``jxf_block_allreduce`` (device copies and
  one reduction kernel);
- ``DistSlab``: one block per rank of a torch.distributed process group
  (NCCL on GPUs), the halo planes sent point to point to the neighbouring
  ranks and the record reduced with all-reduce (max / sum).

``halo_exchange`` and ``allreduce_record`` are written against plain
tensors so that the same code runs over gloo on the CPU (tests) and NCCL.
"""
from __future__ import annotations

import numpy as np

from . import (JXF_HALO_AUX, JXF_HALO_STATE, JXF_PHASE_AUX, JXF_PHASE_FINISH, JXF_PHASE_REDUCE,
               JXF_PHASE_STAGE, JXF_RECORD_LEN, jxf_block, jxf_block_allreduce, jxf_block_exchange,
               jxf_block_halo, jxf_block_halo_count, jxf_block_phase, jxf_block_record,
               jxf_create_block, jxf_destroy, jxf_get_primitive, jxf_get_state, jxf_nvar,
               jxf_set_primitive, jxf_set_state, jxf_stats, structs_from_case)


# ------------------------------------------------------------- host logic --
def slab_blocks(n, ndim: int, nblocks: int, periodic: bool):
    """Equal slabs of the last active axis: per block (lo, n, (lo side
    shared, hi side shared)); a periodic axis wraps the last block to the
    first.  Each block must own at least three planes (the halo depth)."""
    ax = ndim - 1
    N = int(n[ax])
    if nblocks < 1 or N % nblocks:
        raise ValueError("%d cells along the split axis do not split into %d equal blocks" % (N, nblocks))
    m = N // nblocks
    if m < 3:
        raise ValueError("a block needs at least 3 planes along the split axis (got %d)" % m)
    out = []
    for k in range(nblocks):
        lo = [0, 0, 0]
        nn = [int(n[e]) if e < ndim else 1 for e in range(3)]
        lo[ax], nn[ax] = k * m, m
        out.append((lo, nn, (k > 0 or periodic, k < nblocks - 1 or periodic)))
    return out


def neighbour_ranks(rank: int, world: int, shared):
    """Ranks holding the blocks below and above ``rank`` (None where the
    side is a boundary of the grid)."""
    lo = (rank - 1) % world if shared[0] else None
    hi = (rank + 1) % world if shared[1] else None
    return lo, hi


def block_struct(lo, n, shared, ndim: int) -> jxf_block:
    b = jxf_block()
    for e in range(3):
        b.lo[e], b.n[e] = lo[e], n[e]
        b.nbr[e][0] = b.nbr[e][1] = 0
    b.nbr[ndim - 1][0], b.nbr[ndim - 1][1] = int(shared[0]), int(shared[1])
    return b


def split_axis_of_array(ndim: int) -> int:
    """Axis of a state array [v][z][y][x] that the blocks split."""
    return 4 - ndim


def halo_exchange(regions, rank: int, world: int, shared, group=None):
    """Move halo planes between neighbouring ranks.  ``regions``: list of
    {"send": (low-side view, high-side view), "recv": (low, high)} tensors of
    equal shapes (rows x plane values).  Upward transfers (my high side to
    the next rank's low halo) are posted before downward ones, on every rank,
    so that the point-to-point messages between a pair of ranks pair up in
    order even when two ranks are neighbours on both sides (a periodic axis
    over two ranks).  A rank that is its own neighbour copies locally."""
    import torch
    import torch.distributed as dist
    lo, hi = neighbour_ranks(rank, world, shared)
    ops, landing = [], []
    for direction in ("up", "down"):
        for r in regions:
            if direction == "up":
                src, dst_rank, recv_view, recv_rank = r["send"][1], hi, r["recv"][0], lo
            else:
                src, dst_rank, recv_view, recv_rank = r["send"][0], lo, r["recv"][1], hi
            if dst_rank is not None and dst_rank == rank:  # a single rank, periodic
                recv_view.copy_(src)
                continue
            if dst_rank is not None:
                ops.append(dist.P2POp(dist.isend, src.contiguous(), dst_rank, group=group))
            if recv_rank is not None:
                buf = torch.empty(recv_view.shape, dtype=recv_view.dtype, device=recv_view.device)
                ops.append(dist.P2POp(dist.irecv, buf, recv_rank, group=group))
                landing.append((recv_view, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for view, buf in landing:
        view.copy_(buf)


def allreduce_record(record, nv: int, group=None):
    """Reduce a block record over all ranks in place: maximum CFL rate,
    minimum density, any non-admissible block, sum of the conservation
    sums (the time-step and diagnostics all-reduce of Alg. 1)."""
    import torch.distributed as dist
    head = record[:3].clone()
    head[1] = -head[1]
    dist.all_reduce(head, op=dist.ReduceOp.MAX, group=group)
    head[1] = -head[1]
    sums = record[3:3 + nv].clone()
    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    record[:3] = head
    record[3:3 + nv] = sums


# ------------------------------------------------------------ device views --
class _DeviceRegion:
    """A strided region of device memory as a CUDA array interface."""

    def __init__(self, ptr: int, shape, strides, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "strides": tuple(strides),
                                         "typestr": typestr, "data": (int(ptr), False), "version": 2}


def _view(ptr: int, rows: int, cols: int, row_stride_bytes: int, esize: int):
    import torch
    typestr = "<f8" if esize == 8 else "<f4"
    return torch.as_tensor(_DeviceRegion(ptr, (rows, cols), (row_stride_bytes, esize), typestr), device="cuda")


def _regions(h, kind: int, esize: int):
    out = []
    for i in range(jxf_block_halo_count(h, kind)):
        views = {}
        for recv in (0, 1):
            pair = []
            for side in (0, 1):
                ptr, pitch, width, rows = jxf_block_halo(h, kind, i, side, recv)
                pair.append(_view(ptr, rows, width // esize, pitch, esize))
            views["recv" if recv else "send"] = tuple(pair)
        out.append(views)
    return out


# ------------------------------------------------------- one process, many --
class SlabGrid:
    """A workload's grid split into ``nblocks`` slabs, all on the current
    CUDA device, stepped together (same arithmetic as one grid)."""

    def __init__(self, case: dict, precision: str = "fp64", nblocks: int = 2):
        self.case, self.precision, self.ndim = case, precision, case["ndim"]
        self.periodic = case["bc"][self.ndim - 1][0] == "periodic"
        g, e, s = structs_from_case(case, precision)
        self.parts = slab_blocks(case["n"], self.ndim, nblocks, self.periodic)
        self.h = [jxf_create_block(g, e, s, block_struct(lo, n, sh, self.ndim)) for lo, n, sh in self.parts]
        self.nv = jxf_nvar(self.h[0])

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    def close(self):
        for h in getattr(self, "h", []):
            jxf_destroy(h)
        self.h = []

    def _split(self, A):
        ax = split_axis_of_array(self.ndim)
        return np.split(np.asarray(A), len(self.h), axis=ax)

    def _exchange(self, kind):
        nb = len(self.h)
        for k in range(nb):
            if k < nb - 1 or self.periodic:
                jxf_block_exchange(self.h[k], self.h[(k + 1) % nb], kind)

    def _complete(self, mode: int):
        self._exchange(JXF_HALO_STATE)
        for h in self.h:
            jxf_block_phase(h, JXF_PHASE_AUX)
        self._exchange(JXF_HALO_AUX)
        for h in self.h:
            jxf_block_phase(h, JXF_PHASE_REDUCE)
        jxf_block_allreduce(self.h)
        for h in self.h:
            jxf_block_phase(h, JXF_PHASE_FINISH, mode)

    def set_primitive(self, W):
        for h, Wk in zip(self.h, self._split(np.ascontiguousarray(W, dtype=np.float64))):
            jxf_set_primitive(h, np.ascontiguousarray(Wk))
        self._complete(0)

    def set_state(self, U):
        import torch
        ax = split_axis_of_array(self.ndim)
        for h, Uk in zip(self.h, torch.chunk(U, len(self.h), dim=ax)):
            jxf_set_state(h, Uk.contiguous())
        self._complete(0)

    def step(self, n: int):
        for _ in range(n):
            for stage in range(3):
                for h in self.h:
                    jxf_block_phase(h, JXF_PHASE_STAGE, stage)
                self._exchange(JXF_HALO_STATE)
                for h in self.h:
                    jxf_block_phase(h, JXF_PHASE_AUX)
                self._exchange(JXF_HALO_AUX)
            for h in self.h:
                jxf_block_phase(h, JXF_PHASE_REDUCE)
            jxf_block_allreduce(self.h)
            for h in self.h:
                jxf_block_phase(h, JXF_PHASE_FINISH, 1)

    def _gather(self, getter):
        import torch
        parts = []
        for h, (lo, n, _) in zip(self.h, self.parts):
            shape = (self.nv, n[2], n[1], n[0])
            out = torch.empty(shape, dtype=self.dtype, device="cuda")
            getter(h, out)
            parts.append(out)
        return torch.cat(parts, dim=split_axis_of_array(self.ndim))

    def state(self):
        return self._gather(jxf_get_state)

    def primitive(self):
        return self._gather(jxf_get_primitive)

    def stats(self):
        """(conservation sums over the whole grid, last dt, limiter counts
        summed over the blocks)."""
        out = [jxf_stats(h) for h in self.h]
        lim = tuple(int(sum(o[2][k] for o in out)) for k in range(2))
        return out[0][0], out[0][1], lim


# -------------------------------------------------- one block per rank ------
class DistSlab:
    """This rank's block of a grid split over the ranks of a torch.distributed
    group along its last active axis (one block per rank on the rank's
    current CUDA device); halos by point-to-point transfers to the
    neighbouring ranks, the record by all-reduce.  ``case`` describes the
    whole grid (its ``n``, ``dx``, conditions, materials and scheme); its
    ``W`` is not read -- each rank sets its own slab."""

    def __init__(self, case: dict, precision: str = "fp64", group=None):
        import torch.distributed as dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.case, self.precision, self.ndim = case, precision, case["ndim"]
        self.periodic = case["bc"][self.ndim - 1][0] == "periodic"
        self.parts = slab_blocks(case["n"], self.ndim, self.world, self.periodic)
        lo, n, shared = self.parts[self.rank]
        self.shared = shared
        g, e, s = structs_from_case(case, precision)
        self.h = jxf_create_block(g, e, s, block_struct(lo, n, shared, self.ndim))
        self.nv = jxf_nvar(self.h)
        self.esize = 8 if precision == "fp64" else 4
        self.record = _view(jxf_block_record(self.h), 1, JXF_RECORD_LEN, JXF_RECORD_LEN * 8, 8)[0]

    def close(self):
        if getattr(self, "h", None):
            jxf_destroy(self.h)
            self.h = None

    def _exchange(self, kind):
        # the limiter's state region follows the stage: look the regions up each time
        halo_exchange(_regions(self.h, kind, self.esize), self.rank, self.world, self.shared, self.group)

    def _complete(self, mode: int):
        self._exchange(JXF_HALO_STATE)
        jxf_block_phase(self.h, JXF_PHASE_AUX)
        self._exchange(JXF_HALO_AUX)
        jxf_block_phase(self.h, JXF_PHASE_REDUCE)
        allreduce_record(self.record, self.nv, self.group)
        jxf_block_phase(self.h, JXF_PHASE_FINISH, mode)

    def set_primitive(self, W_block):
        """This rank's slab of the primitive field (float64)."""
        jxf_set_primitive(self.h, np.ascontiguousarray(W_block, dtype=np.float64))
        self._complete(0)

    def set_state(self, U_block):
        """This rank's slab of the conservative state (storage type; host or
        device)."""
        jxf_set_state(self.h, U_block)
        self._complete(0)

    def step(self, n: int):
        for _ in range(n):
            for stage in range(3):
                jxf_block_phase(self.h, JXF_PHASE_STAGE, stage)
                self._exchange(JXF_HALO_STATE)
                jxf_block_phase(self.h, JXF_PHASE_AUX)
                self._exchange(JXF_HALO_AUX)
            jxf_block_phase(self.h, JXF_PHASE_REDUCE)
            allreduce_record(self.record, self.nv, self.group)
            jxf_block_phase(self.h, JXF_PHASE_FINISH, 1)

    def state(self):
        import torch
        lo, n, _ = self.parts[self.rank]
        out = torch.empty((self.nv, n[2], n[1], n[0]),
                          dtype=torch.float64 if self.precision == "fp64" else torch.float32, device="cuda")
        jxf_get_state(self.h, out)
        return out

    def stats(self):
        return jxf_stats(self.h)
