"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar (integer and bit work throughout): the GPU lattice equals the DTrDT
replay (O2) bit for bit, the net flip count and the roughness sums S1, S2 are
equal integers, and W^2 is the same double.  Small lattices are compared
whole; L = 2^17 here through properties that hold at any size (exact S1/S2 of
a closed-form lattice, row balance); test_gpu_fullsize.py compares L = 2^17
tile by tile and L = 4096 whole for 16 seeds."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def _oracle_bits(oracle, sim):
    return oracle.unpack_canonical(sim.lattice(), sim.L)


def _assert_same(oracle, sim, X, Y, net=None, what=""):
    Xg, Yg = _oracle_bits(oracle, sim)
    if not (np.array_equal(Xg, X) and np.array_equal(Yg, Y)):
        bad = np.argwhere((Xg != X) | (Yg != Y))
        raise AssertionError(f"{what}: {len(bad)} sites differ, first {bad[:5].tolist()}")
    m = sim.measure()
    s1, s2, hmax = oracle.w2_sums(X, Y)
    assert (m.s1, m.s2, m.hmax) == (s1, s2, hmax), what
    assert m.w2 == oracle.w2_from_sums(sim.L, s1, s2), what
    if net is not None:
        assert m.net_flips == net, what


@pytest.mark.parametrize("L", [64, 192, 256, 1024])
def test_flat_start(g, oracle, L):
    with g.Simulation(L, 1.0, 0.0, 1) as sim:
        X, Y = oracle.flat(L)
        assert np.array_equal(sim.lattice(), oracle.pack_canonical(X, Y))
        assert np.array_equal(sim.planes(), oracle.pack_planar(X, Y))
        m = sim.measure()
        N = L * L
        assert (m.s1, m.s2, m.hmax, m.net_flips, m.w2) == (N // 2, N // 2, 1, 0, 0.25)


def test_kpz_256_bit_exact_through_100_mcs(g, oracle):
    """L = 256, p = 1, q = 0, 64 x 64 sub-tiles, 4 x 4 thread cells, seed 1."""
    prm = oracle.Params(L=256, p=1.0, q=0.0, seed=1, Bx=64, By=64)
    X, Y = oracle.flat(256)
    net = 0
    t = 0
    with g.Simulation(256, 1.0, 0.0, 1, Bx=64, By=64) as sim:
        for tt in (1, 2, 3, 5, 10, 20, 50, 100):
            net += oracle.dtrdt_run(X, Y, prm, t, tt - t)[0]
            sim.run(tt - t)
            t = tt
            _assert_same(oracle, sim, X, Y, net, f"t={t}")
        assert sim.t == 100


CONFIGS = [
    dict(L=256, p=0.95, q=0.05, seed=1, Bx=64, By=64, n=6),
    dict(L=256, p=0.5, q=0.5, seed=2, Bx=32, By=16, n=6),
    dict(L=512, p=0.3, q=0.9, seed=3, Bx=256, By=64, n=4),
    dict(L=192, p=0.8, q=0.2, seed=4, Bx=32, By=32, n=5),
    dict(L=64, p=1.0, q=0.0, seed=5, Bx=32, By=16, n=12),
    dict(L=1024, p=0.95, q=0.05, seed=6, Bx=512, By=32, n=3),
    dict(L=2048, p=0.95, q=0.05, seed=7, Bx=1024, By=16, n=2),
    dict(L=512, p=0.0, q=1.0, seed=8, Bx=128, By=128, n=4),
    dict(L=256, p=0.0, q=0.0, seed=9, Bx=64, By=64, n=3),
    dict(L=384, p=1.0, q=1.0, seed=10, Bx=64, By=32, n=4),
    dict(L=256, p=0.999, q=1e-6, seed=2**40 + 11, Bx=128, By=32, n=5),
]


@pytest.mark.parametrize("c", CONFIGS, ids=lambda c: "L{L}_p{p}_q{q}_B{Bx}x{By}".format(**c))
def test_bit_exact_configs(g, oracle, c):
    prm = oracle.Params(L=c["L"], p=c["p"], q=c["q"], seed=c["seed"], Bx=c["Bx"], By=c["By"])
    X, Y = oracle.flat(c["L"])
    with g.Simulation(c["L"], c["p"], c["q"], c["seed"], Bx=c["Bx"], By=c["By"]) as sim:
        net = 0
        for t in range(c["n"]):
            net += oracle.dtrdt_run(X, Y, prm, t, 1)[0]
            sim.run(1)
            _assert_same(oracle, sim, X, Y, net, f"t={t + 1}")


def test_resume_is_bit_identical(g, oracle):
    L, p, q, seed = 256, 0.95, 0.05, 21
    with g.Simulation(L, p, q, seed) as a:
        a.run(7)
        ref = a.lattice()
    with g.Simulation(L, p, q, seed) as b:
        b.run(3)
        snap = b.lattice()
    with g.Simulation(L, p, q, seed) as c:
        c.set_lattice(snap, 3)
        assert c.t == 3
        c.run(4)
        assert np.array_equal(c.lattice(), ref)


def test_window_and_planes_agree_with_lattice(g, oracle):
    L = 512
    with g.Simulation(L, 0.7, 0.3, 5, Bx=128, By=64) as sim:
        sim.run(3)
        X, Y = _oracle_bits(oracle, sim)
        Xp, Yp = g.planes_to_bits(sim.planes(), L)
        assert np.array_equal(X, Xp) and np.array_equal(Y, Yp)
        for wx, wy, W, H in ((0, 0, 64, 32), (500, 490, 40, 50), (13, 7, 512, 3)):
            Xw, Yw = sim.window(wx, wy, W, H)
            ys = (wy + np.arange(H)) % L
            xs = (wx + np.arange(W)) % L
            assert np.array_equal(Xw, X[np.ix_(ys, xs)])
            assert np.array_equal(Yw, Y[np.ix_(ys, xs)])


def test_invalid_calls(g):
    from paper_1705_01022_gb300 import _lib
    with g.Simulation(256, 1.0, 0.0, 1) as sim:
        with pytest.raises(_lib.OctError):
            _lib.oct_set_lattice(sim.h, np.zeros(10, np.uint32), 10, 0)
        with pytest.raises(_lib.OctError):
            _lib.oct_run_mcs(sim.h, -1)
        with pytest.raises(_lib.OctError):
            sim.set_lattice(np.zeros(256 * 256 // 16, np.uint32), -5)


def _tent(L):
    return np.abs(np.arange(L) - L // 2).astype(np.int64)


def _tent_lattice_planes(L):
    """h(x,y) = tent(x) + tent(y), tent(x) = |x - L/2|: a valid periodic slope
    field with heights of order L; returns planar words."""
    tent = _tent(L)
    up = (tent - np.roll(tent, 1)) == 1  # slope to the left/lower neighbour is +1
    xrow = np.packbits(up.astype(np.uint8), bitorder="little").view(np.uint32)
    Xplane = np.broadcast_to(xrow, (L, L // 32))
    Yplane = np.where(up[:, None], np.uint32(0xFFFFFFFF), np.uint32(0)) * np.ones((1, L // 32), np.uint32)
    return np.concatenate([Xplane.reshape(-1), Yplane.reshape(-1)]).astype(np.uint32)


def _tent_sums(L):
    a = _tent(L) - L // 2  # heights relative to h(0,0)
    sa, sa2 = int(a.sum()), int((a * a).sum())
    s1 = 2 * L * sa
    s2 = 2 * L * sa2 + 2 * sa * sa
    # extremes of a(x) + a(y) are sums of the extremes of a
    hmax = max(abs(2 * int(a.min())), abs(2 * int(a.max())))
    return s1, s2, hmax


@pytest.mark.parametrize("L", [256, 4096])
def test_roughness_of_closed_form_lattice(g, oracle, L):
    words = _tent_lattice_planes(L)
    s1, s2, hmax = _tent_sums(L)
    assert oracle.w2_sums_planar(words, L) == (s1, s2, hmax)
    with g.Simulation(L, 1.0, 0.0, 1) as sim:
        g._lib.oct_set_planes(sim.h, words, words.size, 0)
        m = sim.measure()
        assert (m.s1, m.s2, m.hmax) == (s1, s2, hmax)


def test_c3_full_size_properties(g, oracle):
    """L = 2^17 (1.7e10 sites, 4 GiB), p = 0.95, q = 0.05, 256 x 64 sub-tiles,
    after three MCS: L/2 up-slopes in every row, exact roughness of the evolved
    lattice against the oracle's O3, and the 128-bit S2 of the closed-form
    lattice.  (Tile-by-tile parity at this size: test_gpu_fullsize.py.)"""
    L, p, q, seed, Bx, By = 2**17, 0.95, 0.05, 1, 256, 64
    with g.Simulation(L, p, q, seed, Bx=Bx, By=By) as sim:
        sim.run(3)
        # row balance at full size (X plane): L/2 up-slopes per row
        planes = sim.planes()
        table = np.array([bin(i).count("1") for i in range(256)], dtype=np.uint8)
        xbytes = planes[: L * (L // 32)].view(np.uint8).reshape(L, L // 8)
        for r0 in range(0, L, 4096):
            counts = table[xbytes[r0:r0 + 4096]].sum(axis=1, dtype=np.int64)
            assert np.all(counts == L // 2), r0
        # exact roughness of the evolved lattice against the oracle
        m = sim.measure()
        s1, s2, hmax = oracle.w2_sums_planar(planes, L)
        assert (m.s1, m.s2, m.hmax) == (s1, s2, hmax)
        # 128-bit S2: the closed-form tent lattice at full size
        words = _tent_lattice_planes(L)
        g._lib.oct_set_planes(sim.h, words, words.size, 0)
        del words
        m = sim.measure()
        assert (m.s1, m.s2, m.hmax) == _tent_sums(L)
        assert m.s2_hi > 0


DB_CONFIGS = [
    dict(L=256, p=1.0, q=0.0, seed=1, Bx=64, By=64, n=5),
    dict(L=256, p=0.95, q=0.0, seed=2, Bx=64, By=64, n=4),
    dict(L=512, p=0.6, q=0.3, seed=3, Bx=256, By=64, n=4),
    dict(L=256, p=0.5, q=0.5, seed=4, Bx=32, By=16, n=5),
    dict(L=192, p=0.95, q=0.05, seed=5, Bx=32, By=32, n=4),
    dict(L=1024, p=0.0, q=1.0, seed=6, Bx=512, By=32, n=3),
]


@pytest.mark.parametrize("c", DB_CONFIGS, ids=lambda c: "DB_L{L}_p{p}_q{q}_B{Bx}x{By}".format(**c))
def test_db_bit_exact(g, oracle, c):
    """DTrDB: single-hit dead border at block level (delayed borders when both
    p and q are non-zero), against the oracle bit for bit."""
    prm = oracle.Params(L=c["L"], p=c["p"], q=c["q"], seed=c["seed"], Bx=c["Bx"], By=c["By"],
                        scheme=oracle.SCHEME_DB)
    X, Y = oracle.flat(c["L"])
    with g.Simulation(c["L"], c["p"], c["q"], c["seed"], Bx=c["Bx"], By=c["By"], scheme=1) as sim:
        net = 0
        for t in range(c["n"]):
            net += oracle.dtrdt_run(X, Y, prm, t, 1)[0]
            sim.run(1)
            _assert_same(oracle, sim, X, Y, net, f"t={t + 1}")


DTR_CONFIGS = [
    dict(L=256, p=1.0, q=0.0, seed=1, Bx=64, By=64, n=5),       # 2 x 4 groups per sub-tile
    dict(L=512, p=0.95, q=0.05, seed=2, Bx=256, By=64, n=4),    # a full warp of groups
    dict(L=256, p=0.5, q=0.5, seed=3, Bx=32, By=16, n=6),       # one group: both wraps inside a lane
    dict(L=384, p=0.6, q=0.3, seed=4, Bx=32, By=64, n=4),       # one group column
    dict(L=512, p=0.0, q=0.9, seed=5, Bx=128, By=16, n=4),      # one group row
    dict(L=192, p=0.95, q=0.05, seed=6, Bx=96, By=32, n=5),     # three group columns
]


@pytest.mark.parametrize("c", DTR_CONFIGS, ids=lambda c: "DTR_L{L}_p{p}_q{q}_B{Bx}x{By}".format(**c))
def test_dtr_bit_exact(g, oracle, c):
    """DTrDTr: double tiling with a block-layer origin that moves after every
    collective step (the cell grid wrapping around the sub-tile), against the
    oracle bit for bit."""
    prm = oracle.Params(L=c["L"], p=c["p"], q=c["q"], seed=c["seed"], Bx=c["Bx"], By=c["By"],
                        scheme=oracle.SCHEME_DTR)
    X, Y = oracle.flat(c["L"])
    with g.Simulation(c["L"], c["p"], c["q"], c["seed"], Bx=c["Bx"], By=c["By"],
                      scheme=g._lib.OCT_SCHEME_DTR) as sim:
        net = 0
        for t in range(c["n"]):
            net += oracle.dtrdt_run(X, Y, prm, t, 1)[0]
            sim.run(1)
            _assert_same(oracle, sim, X, Y, net, f"t={t + 1}")


def _all_shapes():
    from paper_1705_01022_gb300 import autotune
    return autotune.candidates(2048)


@pytest.mark.parametrize("shape", _all_shapes(), ids=lambda s: f"{s[0]}x{s[1]}")
def test_every_tunable_shape_bit_exact(g, oracle, shape):
    """Every sub-tile shape the autotuner may choose (at L = 2048: one group up
    to 32, packed several to a warp below 32), both acceptance modes."""
    Bx, By = shape
    for (p, q, seed) in ((0.95, 0.05, 21), (1.0, 0.0, 22)):
        prm = oracle.Params(L=2048, p=p, q=q, seed=seed, Bx=Bx, By=By)
        X, Y = oracle.flat(2048)
        net = oracle.dtrdt_run(X, Y, prm, 0, 2)[0]
        with g.Simulation(2048, p, q, seed, Bx=Bx, By=By) as sim:
            sim.run(2)
            _assert_same(oracle, sim, X, Y, net, f"{Bx}x{By} p={p}")


@pytest.mark.parametrize("L,Bx,By", [(192, 32, 32), (4160, 32, 32), (4224, 64, 64),
                                      (16448, 32, 32), (16512, 64, 64)])
def test_roughness_on_ragged_rows(g, oracle, L, Bx, By):
    """The W^2 row pass (chunks of 512 words, 16 per lane) on rows of 6 words
    (scalar loads), 130 and 132 words (one partial chunk, scalar and 16-byte
    loads), 514 words (a full chunk, then 2 words on scalar loads) and 516
    words (a full chunk, then 4 words on 16-byte loads): S1, S2 and hmax of the
    GPU lattice equal the oracle's O3 on the same lattice, after a few MCS of
    rough dynamics (EW, then KPZ-like)."""
    for p, q, n in ((0.5, 0.5, 3), (0.95, 0.05, 5)):
        with g.Simulation(L, p, q, 77, Bx=Bx, By=By) as sim:
            sim.run(n)
            m = sim.measure()
            X, Y = _oracle_bits(oracle, sim)
            s1, s2, hmax = oracle.w2_sums(X, Y)
            assert (m.s1, m.s2, m.hmax) == (s1, s2, hmax), (L, p, q)
            assert m.w2 == oracle.w2(X, Y)
