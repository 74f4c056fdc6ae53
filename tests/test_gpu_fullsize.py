"""Full-size parity at L = 2^17 (1.7e10 sites, 4 GiB): the first two MCS on
thousands of device tiles, and the 16 seeds of L = 4096 through 20 MCS.

L = 2^17, p = 0.95, q = 0.05, 256 x 64-site sub-tiles (device tiles of
512 x 128 sites, 256 x 1024 of them): for MCS 0 (from the flat start) and
MCS 1 (from the GPU's lattice after MCS 0), bands of full rows are read from
the GPU before and after the MCS.  Windows of 64 x 8 device tiles are cut
from each band and replayed by the oracle (O2 on a window); the interior 60 x
4 device tiles of every window, which no update from outside the window can
reach within one MCS, must equal the GPU's bit for bit.  Two bands of five
windows per MCS give 2400 device tiles per MCS; the first band wraps the
lattice's y edge and the first window of each band its x edge.  DTrDT at 4x4,
8x8 and 16x16-site cells, DTrDB with delayed borders and DTrDTr are checked.
DTrDT at 4x4 cells is also checked on 1024 x 16-site sub-tiles (device tiles
of 2048 x 32 sites), the benchmark's shape: windows of 16 x 32 device tiles
(the same 32768 x 1024 sites) with 12 x 28 interior tiles, 3360 per MCS.

L = 4096 (configuration with 16 seeds): KPZ and EW (p = q = 1/2) through 20
MCS, whole lattices, net flips and roughness sums."""
import multiprocessing as mp

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

L = 2**17
P, Q, SEED = 0.95, 0.05, 1
WINDOWS_PER_BAND = 5


class Geom:
    """Sub-tile Bx x By and a window of (NX + 4) x (NY + 4) device tiles with
    NX x NY interior tiles (two device tiles of margin on every side: within
    one MCS an update reaches at most one sub-tile further per device step)."""

    def __init__(self, Bx, By, NX, NY):
        self.BX, self.BY, self.NX, self.NY = Bx, By, NX, NY
        self.TW, self.TH = 2 * Bx, 2 * By
        self.WIN_W, self.WIN_H = (NX + 4) * self.TW, (NY + 4) * self.TH


G256 = Geom(256, 64, 60, 4)
G1024 = Geom(1024, 16, 12, 28)


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


@pytest.fixture(scope="module")
def pool():
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as p:
        yield p


def _flat_band(y0, H):
    ys = (y0 + np.arange(H)) % L
    xs = np.arange(L)
    b = ((ys[:, None] + xs[None, :]) & 1).astype(np.uint8)  # flat start h = (x+y) mod 2
    return b, b.copy()


def _layout(oracle, prm, t, gm):
    """Band rows and window columns of MCS t: bands start two device tiles
    above their first interior tile row; the first band's interior straddles
    the y edge, the first window's the x edge."""
    ox, oy, _ = oracle.mcs_draw(prm, t)
    TX, TY = L // gm.TW, L // gm.TH
    rng = np.random.default_rng(1000 + t)
    band_t0 = [TY - gm.NY // 2, int(rng.integers(0, TY))]
    win_t0 = [TX - gm.NX // 2] + [int(v) for v in rng.choice(np.arange(TX), WINDOWS_PER_BAND - 1, replace=False)]
    bands = [(oy + gm.TH * (ty0 - 2)) % L for ty0 in band_t0]
    wins = [(ox + gm.TW * (tx0 - 2)) % L for tx0 in win_t0]
    return bands, wins


def _cut(band, wx, gm):
    xs = (wx + np.arange(gm.WIN_W)) % L
    return np.ascontiguousarray(band[:, xs])


def _check_mcs(oracle, pool, sim, prm, t, gm, pre_bands=None):
    """Replays MCS t on the windows of the layout of MCS t and compares their
    interiors with the GPU after the MCS.  pre_bands: the bands before the MCS
    (None: the flat start)."""
    bands, wins = _layout(oracle, prm, t, gm)
    if pre_bands is None:
        pre_bands = [_flat_band(y0, gm.WIN_H) for y0 in bands]
    TW, TH, NX, NY = gm.TW, gm.TH, gm.NX, gm.NY
    inner = (2 * TH, (2 + NY) * TH, 2 * TW, (2 + NX) * TW)
    pdict = dict(L=prm.L, p=prm.p, q=prm.q, seed=prm.seed, Bx=prm.Bx, By=prm.By, cx=prm.cx, cy=prm.cy,
                 scheme=prm.scheme)
    jobs = []
    for y0, (Xb, Yb) in zip(bands, pre_bands):
        for wx in wins:
            jobs.append((pdict, t, wx, y0, _cut(Xb, wx, gm), _cut(Yb, wx, gm), inner))
    sim.run(1)
    want = pool.map(oracle_jobs().window_mcs, jobs)
    i = 0
    for y0 in bands:
        Xg, Yg = sim.window(0, y0, L, gm.WIN_H)
        for wx in wins:
            gx = _cut(Xg, wx, gm)[inner[0]:inner[1], inner[2]:inner[3]]
            gy = _cut(Yg, wx, gm)[inner[0]:inner[1], inner[2]:inner[3]]
            ex, ey = want[i]
            if not (np.array_equal(gx, ex) and np.array_equal(gy, ey)):
                bad = np.argwhere((gx != ex) | (gy != ey))
                raise AssertionError(f"MCS {t}, window ({wx}, {y0}): {len(bad)} sites differ, first {bad[:4].tolist()}")
            i += 1
    return len(jobs) * NX * NY


def oracle_jobs():
    from oracle import jobs
    return jobs


CASES = [("DT_4x4", 0, 4, 4, G256), ("DB_4x4", 1, 4, 4, G256), ("DTR_4x4", 3, 4, 4, G256),
         ("DT_8x8", 0, 8, 8, G256), ("DT_16x16", 0, 16, 16, G256), ("DT_4x4_1024x16", 0, 4, 4, G1024)]


@pytest.mark.parametrize("name,scheme,cx,cy,gm", CASES, ids=[c[0] for c in CASES])
def test_first_two_mcs_on_thousands_of_tiles(g, oracle, pool, name, scheme, cx, cy, gm):
    g_scheme = {0: 0, 1: g._lib.OCT_SCHEME_DB, 3: g._lib.OCT_SCHEME_DTR}[scheme]
    prm = oracle.Params(L=L, p=P, q=Q, seed=SEED, Bx=gm.BX, By=gm.BY, cx=cx, cy=cy, scheme=scheme)
    with g.Simulation(L, P, Q, SEED, Bx=gm.BX, By=gm.BY, cx=cx, cy=cy, scheme=g_scheme) as sim:
        n0 = _check_mcs(oracle, pool, sim, prm, 0, gm)
        # MCS 1 from the GPU's own lattice after MCS 0, read on the bands of MCS 1's layout
        bands, _ = _layout(oracle, prm, 1, gm)
        pre = [sim.window(0, y0, L, gm.WIN_H) for y0 in bands]
        n1 = _check_mcs(oracle, pool, sim, prm, 1, gm, pre)
        assert n0 >= 1000 and n1 >= 1000
        print(f"{name}: {n0} + {n1} device tiles bit-exact")


def test_c2_sixteen_seeds_twenty_mcs(g, oracle, pool):
    """L = 4096 (16.8M sites, 4 MiB), 16 seeds, 64 x 64 sub-tiles: KPZ and EW
    (p = q = 0.5) through 20 MCS, whole lattices against the oracle."""
    jobs_list = [(4096, 1.0, 0.0, s, 64, 64, 20) for s in range(1, 17)]
    jobs_list += [(4096, 0.5, 0.5, s, 64, 64, 20) for s in range(1, 17)]
    results = pool.map(oracle_jobs().dtrdt_final_canonical, jobs_list)
    for (Ls, p, q, seed, Bx, By, n), (words, net, (s1, s2)) in zip(jobs_list, results):
        with g.Simulation(Ls, p, q, seed, Bx=Bx, By=By) as sim:
            sim.run(n)
            assert np.array_equal(sim.lattice(), words), (p, q, seed)
            m = sim.measure()
            assert (m.net_flips, m.s1, m.s2) == (net, s1, s2), (p, q, seed)
