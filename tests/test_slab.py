"""Domain decomposition into slabs of rows (paper_2101_06187_gb300/slab.py):
the row bookkeeping, and the exchange protocol over two and three gloo ranks
on the CPU.  Each rank advances its slab (the interior rows plus H halo rows
a side) with the FP64 oracle standing in for the GPU step and exchanges its
edge rows through the library's TorchTransport; the ranks' interiors,
stitched in rank order, must equal the whole lattice advanced by the oracle
(the step is local in space, so to round-off: the same arithmetic per node).
The force of each rank is the whole lattice's, at the global rows the
bookkeeping assigns to its local rows."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads
from paper_2101_06187_gb300 import slab

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

NX, NY, TAU = 24, 30, 0.7
FORCING = dict(kmin=1, kmax=3, amp=2e-4, seed=97, redraw=4)


def test_partition_covers_the_rows_once():
    for ny, world in ((30, 2), (31, 3), (8, 8), (4096, 7)):
        parts = slab.partition(ny, world)
        assert parts[0][0] == 0 and parts[-1][1] == ny
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
        sizes = [b - a for a, b in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab.partition(3, 4)


def test_slab_rows_bookkeeping():
    r = slab.SlabRows(ny=10, world=3, rank=0, halo=2)
    assert r.rows == (0, 4) and r.ny_ext == 8 and r.prev == 2 and r.next == 1
    assert list(r.global_rows()) == [8, 9, 0, 1, 2, 3, 4, 5]
    g = r.global_rows()
    assert list(g[slice(*r.interior)]) == [0, 1, 2, 3]
    assert list(g[slice(*r.send_up)]) == [2, 3] and list(g[slice(*r.send_down)]) == [0, 1]
    assert list(g[slice(*r.recv_below)]) == [8, 9] and list(g[slice(*r.recv_above)]) == [4, 5]
    # what a rank receives is what its neighbour sends
    for world in (1, 2, 3):
        rows = [slab.SlabRows(31, world, k, 2) for k in range(world)]
        for k, rk in enumerate(rows):
            below, above = rows[rk.prev], rows[rk.next]
            gk = rk.global_rows()
            assert list(gk[slice(*rk.recv_below)]) == list(below.global_rows()[slice(*below.send_up)])
            assert list(gk[slice(*rk.recv_above)]) == list(above.global_rows()[slice(*above.send_down)])
    with pytest.raises(ValueError):
        slab.SlabRows(ny=4, world=4, rank=0, halo=2).check()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_run(rank, world, port, halo, nsteps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_threads(1)
    rows = slab.SlabRows(NY, world, rank, halo)
    rows.check()
    g = rows.global_rows()
    eps, vx, vy = workloads.random_smooth(NX, NY, seed=5, deps=0.05, vmax=0.05)
    f = oracle.init(NX, rows.ny_ext, eps[g], vx[g], vy[g])
    nbytes = 26 * halo * NX * 8
    bufs = [torch.empty(nbytes // 8, dtype=torch.float64) for _ in range(4)]

    def pack(lo, hi, buf):
        buf.copy_(torch.from_numpy(np.ascontiguousarray(f[:, lo:hi, :]).ravel()))

    def unpack(lo, hi, buf):
        f[:, lo:hi, :] = buf.numpy().reshape(26, hi - lo, NX)

    xs = np.tile(np.arange(NX), rows.ny_ext)
    ys = np.repeat(g, NX)
    transport = slab.TorchTransport()
    for s in range(nsteps):
        if s % halo == 0:
            slab.exchange(rows, pack, unpack, transport, bufs)
        Fx, Fy = oracle.force_points(NX, NY, FORCING["kmin"], FORCING["kmax"], FORCING["amp"], FORCING["seed"],
                                     s // FORCING["redraw"], xs, ys)
        oracle.step(f, TAU, Fx.reshape(rows.ny_ext, NX), Fy.reshape(rows.ny_ext, NX))
    out[rank] = np.ascontiguousarray(f[:, slice(*rows.interior), :])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,halo,nsteps", [(2, 1, 9), (2, 2, 10), (3, 1, 7)])
def test_slabs_over_gloo_ranks_equal_the_whole_lattice(world, halo, nsteps):
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_run, args=(world, _free_port(), halo, nsteps, out), nprocs=world, join=True)
    got = np.concatenate([out[r] for r in range(world)], axis=1)
    eps, vx, vy = workloads.random_smooth(NX, NY, seed=5, deps=0.05, vmax=0.05)
    ref = oracle.init(NX, NY, eps, vx, vy)
    oracle.run(ref, TAU, nsteps, kmin=FORCING["kmin"], kmax=FORCING["kmax"], amp=FORCING["amp"],
               seed=FORCING["seed"], redraw=FORCING["redraw"])
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_exchange_without_refresh_corrupts_the_edges():
    """The halo exchange is what keeps the slabs right: skipping it lets the
    wrapped slab's garbage reach the interior after more than H steps (a
    check that the stitched comparison above can fail)."""
    world, halo, nsteps = 1, 1, 3
    rows = slab.SlabRows(NY // 2, world, 0, halo)   # half the lattice as if it were whole: wrong neighbours
    g = np.arange(-halo, NY // 2 + halo) % NY
    eps, vx, vy = workloads.random_smooth(NX, NY, seed=5, deps=0.05, vmax=0.05)
    f = oracle.init(NX, rows.ny_ext, eps[g], vx[g], vy[g])
    for _ in range(nsteps):
        oracle.step(f, TAU)
    ref = oracle.init(NX, NY, eps, vx, vy)
    oracle.run(ref, TAU, nsteps)
    diff = np.abs(f[:, slice(*rows.interior), :] - ref[:, : NY // 2, :])
    assert np.max(diff) > 1e-6
