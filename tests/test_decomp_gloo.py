"""The decomposed grid's host logic on the CPU (§4.2, §4.3, Alg. 1): slab
split and neighbours, the halo exchange between ranks and the all-reduce of
the block records, run as gloo process groups of world size 1 and 2 on
plain tensors laid out as the library lays out a block (three halo planes
before and after the owned planes of each variable)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2402_05193_gb300 import decomp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_blocks_split_and_neighbours():
    parts = decomp.slab_blocks([16, 12, 24], 3, 4, periodic=False)
    assert [p[0][2] for p in parts] == [0, 6, 12, 18] and all(p[1] == [16, 12, 6] for p in parts)
    assert [p[2] for p in parts] == [(False, True), (True, True), (True, True), (True, False)]
    per = decomp.slab_blocks([16, 12, 24], 3, 2, periodic=True)
    assert [p[2] for p in per] == [(True, True), (True, True)]
    assert decomp.neighbour_ranks(0, 2, (True, True)) == (1, 1)
    assert decomp.neighbour_ranks(0, 4, (False, True)) == (None, 1)
    assert decomp.neighbour_ranks(3, 4, (True, False)) == (2, None)
    assert decomp.neighbour_ranks(3, 4, (True, True)) == (2, 0)
    two_d = decomp.slab_blocks([20, 9], 2, 3, periodic=False)  # 2-D grids split along y
    assert [p[0][1] for p in two_d] == [0, 3, 6] and two_d[0][1] == [20, 3, 1]
    assert decomp.split_axis_of_array(3) == 1 and decomp.split_axis_of_array(2) == 2
    with pytest.raises(ValueError):
        decomp.slab_blocks([8, 8, 10], 3, 4, periodic=True)  # not equal blocks
    with pytest.raises(ValueError):
        decomp.slab_blocks([8, 8, 8], 3, 4, periodic=True)  # fewer than 3 planes per block


def _block_arrays(rank, m, plane, rows, N):
    """Padded rows of one block: owned plane z holds rows*1e6 + global plane
    index * plane + offset in the plane; halos hold NaN."""
    A = torch.full((rows, (m + 6) * plane), float("nan"), dtype=torch.float64)
    for r in range(rows):
        for z in range(m):
            g = rank * m + z
            A[r, (z + 3) * plane:(z + 4) * plane] = r * 1e6 + g * plane + torch.arange(plane, dtype=torch.float64)
    return A


def _regions(A, m, plane):
    w = 3 * plane
    return [{"send": (A[:, 3 * plane:3 * plane + w], A[:, m * plane:m * plane + w]),
             "recv": (A[:, 0:w], A[:, (m + 3) * plane:(m + 3) * plane + w])}]


def _expected(r, g, plane, N, periodic):
    if not periodic and (g < 0 or g >= N):
        return None
    return r * 1e6 + (g % N) * plane + np.arange(plane)


def _worker(rank, world, port, periodic, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, plane, rows = 4, 6, 3
    N = m * world
    parts = decomp.slab_blocks([3, 2, N], 3, world, periodic)
    shared = parts[rank][2]
    A = _block_arrays(rank, m, plane, rows, N)
    decomp.halo_exchange(_regions(A, m, plane), rank, world, shared)
    # the record: [max rate, min density, flag, sums...]
    rec = torch.zeros(10, dtype=torch.float64)
    rec[0], rec[1], rec[2] = 1.0 + rank, 0.5 - 0.1 * rank, float(rank == world - 1 and world > 1)
    rec[3:8] = torch.arange(5, dtype=torch.float64) * (rank + 1)
    decomp.allreduce_record(rec, 5)
    out.put((rank, A.numpy(), rec.numpy()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world, periodic", [(2, True), (2, False), (1, True)])
def test_halo_exchange_and_record_allreduce_over_gloo(world, periodic):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m, plane, rows = 4, 6, 3
    N = m * world
    for rank, A, rec in res:
        for r in range(rows):
            for k in range(3):  # halo planes: global planes lo-3..lo-1 and lo+m..lo+m+2
                for g, col in ((rank * m - 3 + k, k), (rank * m + m + k, m + 3 + k)):
                    got = A[r, col * plane:(col + 1) * plane]
                    exp = _expected(r, g, plane, N, periodic)
                    if exp is None:
                        assert np.all(np.isnan(got)), (rank, r, g)
                    else:
                        assert np.array_equal(got, exp), (rank, r, g, got, exp)
        # record: identical on every rank, max / min / any / sum
        assert rec[0] == float(world) and abs(rec[1] - (0.5 - 0.1 * (world - 1))) < 1e-15
        assert rec[2] == (1.0 if world > 1 else 0.0)
        assert np.array_equal(rec[3:8], np.arange(5) * sum(range(1, world + 1)))
