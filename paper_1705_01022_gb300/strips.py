"""One lattice split into row strips over several devices (ranks).

DTr tiles the lattice with device tiles of 2Bx x 2By sites at a random origin
(Sec. 3, Fig. 2); whether a tile belongs to one strip or another only depends
on the origin modulo 2By.  Rank r of n owns the rows [r H, (r+1) H), H = L/n a
multiple of 2By, and updates the device-tile rows whose first row lies there.
Such a tile's sub-tiles reach at most 2By rows past the strip (a sub-tile and
its +y halo row), so a rank holds its strip and the first 2By rows of the next
strip (periodic: rank n-1's are rank 0's first rows).  Per device step:

* before it, the rank's halo rows are refreshed from the next rank (its first
  2By rows);
* after it, the rows of the next strip the rank may have changed, the first
  ((oy - row0) mod 2By) + By*sy - By + 1 of them for sub-tile set sy, go back
  to the next rank.  No row is changed by two ranks in one device step (the
  sub-tiles of one set are 2By rows apart), so overwriting is exact.

Every attempt uses the random streams of the whole lattice (tile index T of
the whole lattice), so the split run is bit-identical to the single-device
run.  W^2 is combined exactly from per-strip partial sums (oct_strip_combine).

The halo moves by torch.distributed point-to-point sends of plain buffers
(NCCL between GPUs, gloo on the host); no peer memory is handed to any kernel.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import _lib


@dataclass(frozen=True)
class StripLayout:
    L: int
    By: int
    nranks: int
    rank: int

    def __post_init__(self):
        if self.L % self.nranks or (self.L // self.nranks) % (2 * self.By):
            raise ValueError("L / nranks must be a multiple of 2 By")
        if not 0 <= self.rank < self.nranks:
            raise ValueError("rank outside 0 .. nranks-1")

    @property
    def H(self) -> int:
        """Rows the strip owns."""
        return self.L // self.nranks

    @property
    def row0(self) -> int:
        return self.rank * self.H

    @property
    def halo(self) -> int:
        return 2 * self.By

    @property
    def held(self) -> int:
        """Rows the rank holds: its strip and the next strip's first 2By rows."""
        return self.H + self.halo

    @property
    def next_rank(self) -> int:
        return (self.rank + 1) % self.nranks

    @property
    def prev_rank(self) -> int:
        return (self.rank - 1) % self.nranks

    def changed_below(self, seed: int, t: int, k: int) -> int:
        """Rows of the next strip that device step k of MCS t may change."""
        _, oy, perm = _lib.oct_mcs_draw(seed, self.L, t)
        sy = perm[k] >> 1
        n = (oy - self.row0) % (2 * self.By) + self.By * sy - self.By + 1
        return max(0, n)


class HaloExchange:
    """Moves halo rows of planar strip buffers (tensors of shape (2, held,
    L/32): X plane, then Y plane) between neighbouring ranks."""

    def __init__(self, layout: StripLayout, dist=None):
        self.lay = layout
        self.dist = dist

    def _swap(self, send, dst: int, recv, src: int) -> None:
        if self.lay.nranks == 1:
            recv.copy_(send)
            return
        ops = [self.dist.P2POp(self.dist.isend, send, dst), self.dist.P2POp(self.dist.irecv, recv, src)]
        for req in self.dist.batch_isend_irecv(ops):
            req.wait()

    def refresh_halo(self, buf) -> None:
        """Rows [H, H + 2By) := the next rank's rows [0, 2By)."""
        lay = self.lay
        send = buf[:, 0:lay.halo].contiguous()
        recv = send.new_empty(send.shape)
        self._swap(send, lay.prev_rank, recv, lay.next_rank)
        buf[:, lay.H:lay.H + lay.halo].copy_(recv)

    def return_rows(self, buf, n: int) -> None:
        """The next rank's rows [0, n) := this rank's rows [H, H + n) (the rows
        it changed there), and this rank's rows [0, n) from the previous rank."""
        if n <= 0:
            return
        lay = self.lay
        send = buf[:, lay.H:lay.H + n].contiguous()
        recv = send.new_empty(send.shape)
        self._swap(send, lay.next_rank, recv, lay.prev_rank)
        buf[:, 0:n].copy_(recv)


class GpuStripEngine:
    """A strip handle of the CUDA library on an external device buffer."""

    def __init__(self, layout: StripLayout, p: float, q: float, seed: int, Bx: int, cx: int = 0, cy: int = 0,
                 scheme: int = 0, device=None):
        import torch

        from . import Simulation
        self.torch = torch
        self.lay = layout
        wpr = layout.L // 32
        self.buf = torch.empty((2, layout.held, wpr), dtype=torch.int32, device=device or "cuda")
        self.stream = torch.cuda.current_stream(self.buf.device)
        self.sim = Simulation(layout.L, p, q, seed, Bx=Bx, By=layout.By, cx=cx, cy=cy, scheme=scheme,
                              stream=self.stream, lattice=self.buf,
                              strip=(layout.row0, layout.H, layout.held))
        self.seed = seed

    @property
    def t(self) -> int:
        return self.sim.t

    def step(self, k: int) -> None:
        _lib.oct_device_step(self.sim.h, k)

    def end_mcs(self) -> None:
        _lib.oct_end_mcs(self.sim.h)

    def partial(self) -> _lib.oct_strip_sums:
        return _lib.oct_strip_measure(self.sim.h)

    def close(self) -> None:
        self.sim.close()


class StripRunner:
    """Runs MCS of a split lattice: per device step, refresh the halo, step,
    return the changed rows.  `engine` holds the rank's strip buffer as
    `buf` and offers step(k), end_mcs(), partial() and `t`."""

    def __init__(self, layout: StripLayout, engine, seed: int, dist=None):
        self.lay = layout
        self.engine = engine
        self.seed = seed
        self.dist = dist
        self.x = HaloExchange(layout, dist)

    def run(self, n: int) -> None:
        for _ in range(n):
            t = self.engine.t
            for k in range(4):
                self.x.refresh_halo(self.engine.buf)
                self.engine.step(k)
                self.x.return_rows(self.engine.buf, self.lay.changed_below(self.seed, t, k))
            self.engine.end_mcs()

    def measure(self) -> _lib.oct_w2:
        """Exact W^2 of the whole lattice (every rank gets it)."""
        import ctypes

        import torch
        mine = self.engine.partial()
        fields = [f for f, _ in _lib.oct_strip_sums._fields_]
        vals = [int(getattr(mine, f)) for f in fields]
        vec = torch.tensor([v - (1 << 64) if v >= (1 << 63) else v for v in vals], dtype=torch.int64)
        if self.lay.nranks > 1:
            dev = self.engine.buf.device
            parts_t = [torch.empty_like(vec, device=dev) for _ in range(self.lay.nranks)]
            self.dist.all_gather(parts_t, vec.to(dev))
            rows = [p.cpu().tolist() for p in parts_t]
        else:
            rows = [vec.tolist()]
        parts = []
        for r in rows:
            s = _lib.oct_strip_sums()
            for f, v in zip(fields, r):
                setattr(s, f, ctypes.c_uint64(v).value if f == "p2_lo" or f == "p2_hi" else v)
            parts.append(s)
        return _lib.oct_strip_combine(parts)


def run_local(engines, layouts, seed: int, n: int) -> None:
    """Runs n MCS of a lattice split into strips whose engines all live in this
    process (on one device): the same schedule as StripRunner, with the halo
    rows copied between the strips' buffers.  The strips' kernels never wait
    on one another; each device step of every strip is launched after the
    copies it needs, in stream order."""
    m = len(engines)
    for _ in range(n):
        t = engines[0].t
        for k in range(4):
            for r in range(m):  # halo rows := the next strip's first 2By rows
                lay, nxt = layouts[r], engines[(r + 1) % m]
                engines[r].buf[:, lay.H:lay.H + lay.halo].copy_(nxt.buf[:, 0:lay.halo])
            for e in engines:
                e.step(k)
            for r in range(m):  # the rows of the next strip this one changed go back
                lay = layouts[r]
                c = lay.changed_below(seed, t, k)
                if c > 0:
                    engines[(r + 1) % m].buf[:, 0:c].copy_(engines[r].buf[:, lay.H:lay.H + c])
        for e in engines:
            e.end_mcs()


def combine_local(engines) -> _lib.oct_w2:
    """Exact W^2 of a lattice split into strips held in this process."""
    return _lib.oct_strip_combine([e.partial() for e in engines])
