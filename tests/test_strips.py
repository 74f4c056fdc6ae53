"""Row-strip partition of one lattice over several ranks (host logic, no GPU).

* oct_strip_combine (host code of the C library) forms the whole lattice's
  exact S1, S2, hmax and W^2 from per-strip partial sums written out here from
  their definition; it must equal the oracle's O3 on the whole lattice.
* StripLayout.changed_below equals the rows of the next strip that the owned
  sub-tiles touch, enumerated here from the device-layer draw.
* Two and four gloo ranks (processes on the CPU) run the strip schedule with
  the oracle standing in for the kernels (oracle.device_step_strip on each
  rank's held rows) and exchange halos with torch.distributed: the gathered
  lattice equals the oracle's single-lattice replay bit for bit, and the
  combined W^2 equals O3."""
import os
import socket

import numpy as np
import pytest

from paper_1705_01022_gb300 import _lib, strips


def _partial(X, Y, a, H, t=0, net=0):
    """Strip sums of rows [a, a+H) by definition: heights e_j + r_j(x)
    relative to the strip's first row's h(0, .)."""
    L = X.shape[1]
    rows = (a + np.arange(H)) % X.shape[0]
    Xs, Ys = X[rows].astype(np.int64), Y[rows].astype(np.int64)
    steps_y = 2 * Ys[:, 0] - 1
    e = np.concatenate([[0], np.cumsum(steps_y[1:])])
    sx = 2 * Xs - 1
    sx[:, 0] = 0
    r = np.cumsum(sx, axis=1)
    h = e[:, None] + r
    p = _lib.oct_strip_sums()
    p.rows, p.L, p.f, p.e_last = H, L, int(steps_y[0]), int(e[-1])
    p.p1 = int(h.sum())
    p2 = int((h.astype(object) ** 2).sum())
    p.p2_lo, p.p2_hi = p2 & ((1 << 64) - 1), p2 >> 64
    p.lo, p.hi, p.t, p.net_flips = int(h.min()), int(h.max()), t, net
    return p


@pytest.mark.parametrize("cuts", [(64, 64, 64, 64), (32, 96, 128), (256,)])
def test_combine_equals_whole_lattice_roughness(oracle, cuts):
    L = 256
    X, Y = oracle.flat(L)
    oracle.dtrdt_run(X, Y, oracle.Params(L=L, p=0.8, q=0.2, seed=17, Bx=32, By=32), 0, 6)
    parts, a = [], 0
    for H in cuts:
        parts.append(_partial(X, Y, a, H))
        a += H
    _lib.load()
    got = _lib.oct_strip_combine(parts)
    s1, s2, hmax = oracle.w2_sums(X, Y)
    assert (got.s1, got.s2, got.hmax) == (s1, s2, hmax)
    assert got.w2 == oracle.w2(X, Y)


def test_combine_rejects_strips_that_do_not_cover_the_lattice():
    _lib.load()
    p = _lib.oct_strip_sums()
    p.rows, p.L = 64, 256
    with pytest.raises(_lib.OctError):
        _lib.oct_strip_combine([p, p])


def test_changed_rows_below_a_strip(oracle):
    """Rows of the next strip the owned sub-tiles touch (sub-tile rows and the
    +y halo row), enumerated from the device-layer draw."""
    _lib.load()
    L, By, Bx = 512, 32, 64
    for nranks in (2, 4):
        for rank in range(nranks):
            lay = strips.StripLayout(L, By, nranks, rank)
            for t in range(12):
                ox, oy, perm = oracle.mcs_draw(oracle.Params(L=L, p=0.5, q=0.5, seed=9, Bx=Bx, By=By), t)
                for k in range(4):
                    sy = perm[k] >> 1
                    below = 0
                    for ty in range(L // (2 * By)):
                        yt = (oy + 2 * By * ty) % L
                        if (yt - lay.row0) % L >= lay.H:
                            continue
                        top = (yt - lay.row0) % L + By * sy + By  # local row of the halo row
                        below = max(below, top - lay.H + 1)
                    assert lay.changed_below(9, t, k) == below, (nranks, rank, t, k)


# --------------------------------------------------------- gloo ranks ---

def _pack(Xb, Yb):
    rows, L = Xb.shape
    bits = np.stack([Xb, Yb]).astype(np.uint8)
    return np.packbits(bits.reshape(2, rows, L // 8, 8), axis=-1, bitorder="little").reshape(2, rows, L // 32 * 4)


class OracleStripEngine:
    """The oracle standing in for the kernels: device steps of the rank's
    strip on its held rows (test infrastructure)."""

    def __init__(self, lay, prm):
        import torch
        self.lay, self.prm, self.t = lay, prm, 0
        L = prm.L
        rows = (lay.row0 + np.arange(lay.held)) % L
        flat = ((rows[:, None] + np.arange(L)[None, :]) & 1).astype(np.uint8)
        self.buf = torch.from_numpy(_pack(flat, flat).view(np.int32).copy())
        self.net = 0

    def _bits(self):
        b = np.unpackbits(self.buf.numpy().view(np.uint8), axis=-1, bitorder="little")
        return np.ascontiguousarray(b[0]), np.ascontiguousarray(b[1])

    def step(self, k):
        import oracle
        Xs, Ys = self._bits()
        self.net += oracle.device_step_strip(Xs, Ys, self.prm, self.t, k, self.lay.row0, self.lay.H)
        self.buf.copy_(__import__("torch").from_numpy(_pack(Xs, Ys).view(np.int32).copy()))

    def end_mcs(self):
        self.t += 1

    def partial(self):
        Xs, Ys = self._bits()
        return _partial(Xs, Ys, 0, self.lay.H, self.t, self.net)


def _rank_main(rank, world, port, L, By, p, q, seed, n_mcs, scheme, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        _lib.load()
        lay = strips.StripLayout(L, By, world, rank)
        prm = oracle.Params(L=L, p=p, q=q, seed=seed, Bx=2 * By, By=By, scheme=scheme)
        eng = OracleStripEngine(lay, prm)
        run = strips.StripRunner(lay, eng, seed, dist)
        run.run(n_mcs)
        w = run.measure()
        own = eng.buf[:, :lay.H].contiguous()
        gathered = [torch.empty_like(own) for _ in range(world)]
        dist.all_gather(gathered, own)
        if rank == 0:
            full = torch.cat(gathered, dim=1).numpy()
            np.save(os.path.join(out_dir, "lattice.npy"), full)
            np.save(os.path.join(out_dir, "w2.npy"), np.array([w.s1, w.s2, w.hmax, w.net_flips], dtype=object),
                    allow_pickle=True)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,L,scheme", [(2, 256, 0), (4, 512, 0), (2, 256, 1), (2, 256, 3)],
                         ids=["2ranks_DT", "4ranks_DT", "2ranks_DB", "2ranks_DTR"])
def test_ranks_reproduce_the_single_lattice_run(oracle, tmp_path, world, L, scheme):
    import torch.multiprocessing as tmp
    By, p, q, seed, n = 32, 0.95, 0.05, 5, 3
    tmp.spawn(_rank_main, args=(world, _free_port(), L, By, p, q, seed, n, scheme, str(tmp_path)),
              nprocs=world, join=True)
    full = np.load(tmp_path / "lattice.npy")
    X, Y = oracle.flat(L)
    net = oracle.dtrdt_run(X, Y, oracle.Params(L=L, p=p, q=q, seed=seed, Bx=2 * By, By=By, scheme=scheme), 0, n)[0]
    assert np.array_equal(full, _pack(X, Y).view(np.int32))
    s1, s2, hmax = oracle.w2_sums(X, Y)
    got = np.load(tmp_path / "w2.npy", allow_pickle=True)
    assert (int(got[0]), int(got[1]), int(got[2]), int(got[3])) == (s1, s2, hmax, net)
