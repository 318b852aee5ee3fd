"""Domain decomposition of one lattice into slabs of rows.

The step of Sec. 3.3 is local in space: a node's update reads only its 3 x 3
neighbourhood of the previous state (Sec. 3.2's pull at cfl <= 1).  A lattice
of ny rows split into slabs of consecutive rows therefore advances exactly
like the whole lattice if every slab carries H halo rows on each side, copied
from its neighbours' edge rows before every H steps.  Each slab is an
ordinary lattice of ny_local + 2 H rows (periodic inside itself); after H
steps its outermost H rows on each side hold garbage, its ny_local interior
rows the whole lattice's values, and the next exchange replaces the garbage.
The stirring force is drawn in the frame of the whole lattice
(rlbm_set_force_frame), so every slab sees its own rows of the same field.

Pieces:
* partition / SlabRows: which global rows each rank owns, which local rows
  it sends and receives, and the global row of every local row;
* Transport: moves the edge rows between neighbouring ranks.  TorchTransport
  runs over torch.distributed point-to-point calls (NCCL with device
  buffers, gloo with host buffers), in two shifts per exchange: every rank
  sends its top rows to the next rank and receives the previous rank's, then
  the same downwards -- one send and one receive per rank and shift, so
  messages match in order on any backend and any world size (2 included,
  where both neighbours are the same rank);
* SlabLattice: one slab on the GPU (a Lattice with the force frame set and
  device halo buffers), exchanging through a transport;
* SlabGroup: several slabs of one lattice in one process, exchanging by
  device copies (a decomposition run end to end on one GPU).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Sequence, Tuple

import numpy as np


def partition(ny: int, world: int) -> List[Tuple[int, int]]:
    """Global rows [y0, y1) of each rank: consecutive slabs whose sizes
    differ by at most one row."""
    if world < 1 or ny < world:
        raise ValueError("cannot split %d rows over %d ranks" % (ny, world))
    base, extra = divmod(ny, world)
    out, y = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((y, y + n))
        y += n
    return out


@dataclass(frozen=True)
class SlabRows:
    """Row bookkeeping of one rank's slab (local rows count from the
    bottom halo: local row i is global row (y0 - halo + i) mod ny)."""
    ny: int        # rows of the whole lattice
    world: int
    rank: int
    halo: int      # H: halo rows per side = steps between exchanges

    @property
    def rows(self) -> Tuple[int, int]:
        return partition(self.ny, self.world)[self.rank]

    @property
    def ny_local(self) -> int:
        y0, y1 = self.rows
        return y1 - y0

    @property
    def ny_ext(self) -> int:
        return self.ny_local + 2 * self.halo

    @property
    def prev(self) -> int:
        return (self.rank - 1) % self.world

    @property
    def next(self) -> int:
        return (self.rank + 1) % self.world

    @property
    def interior(self) -> Tuple[int, int]:
        return self.halo, self.halo + self.ny_local

    @property
    def send_up(self) -> Tuple[int, int]:
        """The top H interior rows: the next rank's bottom halo."""
        return self.ny_local, self.ny_local + self.halo

    @property
    def send_down(self) -> Tuple[int, int]:
        """The bottom H interior rows: the previous rank's top halo."""
        return self.halo, 2 * self.halo

    @property
    def recv_below(self) -> Tuple[int, int]:
        """Bottom halo rows, filled from the previous rank's top rows."""
        return 0, self.halo

    @property
    def recv_above(self) -> Tuple[int, int]:
        """Top halo rows, filled from the next rank's bottom rows."""
        return self.halo + self.ny_local, self.ny_ext

    @property
    def frame_y0(self) -> int:
        """Global row of local row 0 (negative for the first slab's halo)."""
        return self.rows[0] - self.halo

    def global_rows(self) -> np.ndarray:
        """Global row index of every local row, periodic."""
        return (self.frame_y0 + np.arange(self.ny_ext)) % self.ny

    def check(self):
        if self.halo < 1:
            raise ValueError("halo must be >= 1")
        if self.ny_local < self.halo:
            raise ValueError("slabs of %d rows cannot feed %d halo rows" % (self.ny_local, self.halo))


class TorchTransport:
    """Edge-row exchange over torch.distributed point-to-point calls."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def shift(self, send, recv, to_rank: int, from_rank: int):
        """Send `send` to to_rank and receive `recv` from from_rank."""
        dist = self.dist
        ops = [dist.P2POp(dist.isend, send, to_rank, self.group), dist.P2POp(dist.irecv, recv, from_rank, self.group)]
        for w in dist.batch_isend_irecv(ops):
            w.wait()


def exchange(rows: SlabRows, pack: Callable, unpack: Callable, transport, bufs,
             sync: Callable = lambda: None) -> None:
    """One halo exchange of a rank.  pack(lo, hi, buf) copies local rows
    [lo, hi) into buf, unpack(lo, hi, buf) the reverse; bufs holds four
    equal buffers (send_up, send_down, recv_below, recv_above); sync() is
    called once the packed rows must be in their buffers and once the
    received rows must have arrived (a device synchronisation on the GPU)."""
    send_up, send_down, recv_below, recv_above = bufs
    pack(*rows.send_up, send_up)
    pack(*rows.send_down, send_down)
    sync()
    transport.shift(send_up, recv_below, rows.next, rows.prev)    # upwards
    transport.shift(send_down, recv_above, rows.prev, rows.next)  # downwards
    sync()
    unpack(*rows.recv_below, recv_below)
    unpack(*rows.recv_above, recv_above)


class SlabLattice:
    """One rank's slab of an nx x ny lattice on the GPU: a Lattice of
    ny_local + 2 H rows with the stirring force drawn in the whole lattice's
    frame.  halo = H is the number of steps between exchanges (2 lets the
    two-steps-per-launch kernel run between exchanges).  transport: a
    TorchTransport (one slab per process); SlabGroup passes its own."""

    def __init__(self, nx: int, ny: int, tau: float, rank: int, world: int, halo: int = 1, transport=None,
                 **lattice_kw):
        import torch

        from . import Lattice
        self.rows = SlabRows(int(ny), int(world), int(rank), int(halo))
        self.rows.check()
        self.nx, self.ny = int(nx), int(ny)
        self.transport = transport
        self.lat = Lattice(self.nx, self.rows.ny_ext, tau, **lattice_kw)
        self.lat.set_force_frame(self.nx, self.ny, 0, self.rows.frame_y0)
        info = self.lat.info()
        self.pitch = info["pitch"]
        nbytes = info["nclasses"] * self.rows.halo * self.pitch * _storage_bytes(self.lat.dtype)
        dev = torch.device("cuda", self.lat.device)
        self.bufs = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(4)]
        self.steps = 0

    # row copies on the lattice's stream
    def pack(self, lo: int, hi: int, buf) -> None:
        self.lat.halo_pack(lo, hi - lo, buf.data_ptr())

    def unpack(self, lo: int, hi: int, buf) -> None:
        self.lat.halo_unpack(lo, hi - lo, buf.data_ptr())

    def local_fields(self, eps, vx, vy):
        """This slab's rows (halos included) of whole-lattice (ny, nx) fields."""
        g = self.rows.global_rows()
        return tuple(np.ascontiguousarray(np.asarray(a)[g]) for a in (eps, vx, vy))

    def init_fields(self, eps, vx, vy) -> None:
        self.lat.init_fields(*self.local_fields(eps, vx, vy))
        self.steps = 0

    def exchange(self) -> None:
        import torch

        def sync():
            self.lat.synchronize()
            torch.cuda.synchronize(self.lat.device)

        sync()
        exchange(self.rows, self.pack, self.unpack, self.transport, self.bufs, sync)

    def step(self, n: int) -> None:
        """Advance n steps (a multiple of the halo width)."""
        H = self.rows.halo
        if n % H:
            raise ValueError("step counts must be multiples of the halo width %d" % H)
        for _ in range(n // H):
            self.exchange()
            self.lat.step(H)
        self.steps += n

    def interior(self, a):
        lo, hi = self.rows.interior
        return a[lo:hi]

    def moments(self):
        """(eps, vx, vy) of the interior rows, (ny_local, nx) each.  The
        moments are those of the streamed state (what the next collision
        sees), which pulls from the halo rows, so this exchanges first: a
        collective call, made by every rank."""
        self.exchange()
        e, vx, vy, _ = self.lat.moments()
        return self.interior(e), self.interior(vx), self.interior(vy)

    def close(self) -> None:
        self.lat.close()


class SlabGroup:
    """All slabs of one lattice in one process, exchanging by device copies:
    the decomposition run end to end on one GPU (no collectives, so nothing
    waits on another launch).  Results equal the whole lattice's."""

    def __init__(self, nx: int, ny: int, tau: float, world: int, halo: int = 1, **lattice_kw):
        self.slabs = [SlabLattice(nx, ny, tau, r, world, halo, None, **lattice_kw) for r in range(world)]
        self.halo = halo

    def init_fields(self, eps, vx, vy) -> None:
        for s in self.slabs:
            s.init_fields(eps, vx, vy)

    def exchange(self) -> None:
        for s in self.slabs:
            s.lat.synchronize()
        for s in self.slabs:
            send_up, send_down = s.bufs[0], s.bufs[1]
            s.pack(*s.rows.send_up, send_up)
            s.pack(*s.rows.send_down, send_down)
        for s in self.slabs:
            s.lat.synchronize()
        for s in self.slabs:
            below = self.slabs[s.rows.prev]
            above = self.slabs[s.rows.next]
            s.unpack(*s.rows.recv_below, below.bufs[0])  # the previous slab's top rows
            s.unpack(*s.rows.recv_above, above.bufs[1])  # the next slab's bottom rows
        for s in self.slabs:
            s.lat.synchronize()

    def step(self, n: int) -> None:
        H = self.halo
        if n % H:
            raise ValueError("step counts must be multiples of the halo width %d" % H)
        for _ in range(n // H):
            self.exchange()
            for s in self.slabs:
                s.lat.step(H)

    def moments(self):
        """Whole-lattice (eps, vx, vy) stitched from the slabs' interiors
        (after an exchange: the streamed state pulls from the halo rows)."""
        self.exchange()
        parts = []
        for s in self.slabs:
            e, vx, vy, _ = s.lat.moments()
            parts.append((s.interior(e), s.interior(vx), s.interior(vy)))
        return tuple(np.concatenate([p[k] for p in parts], axis=0) for k in range(3))

    def close(self) -> None:
        for s in self.slabs:
            s.close()


def _storage_bytes(dtype: str) -> int:
    return {"f64": 8, "f32": 4, "bf16": 2, "f16": 2}[dtype]


def stitch(parts: Sequence[np.ndarray]) -> np.ndarray:
    """Whole-lattice rows from the ranks' interior rows, in rank order."""
    return np.concatenate(list(parts), axis=0)
