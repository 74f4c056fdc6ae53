"""GPU parity of DTrDT with thread cells coarser than 4x4 sites.

The paper's block-layer configurations run from TC=1,1 (8x8 sites) up to
TC=3,2 (32x16) and TC=1,3 / 3,1 (Sec. 3.1.1 notation; Sec. 4.1.2, Fig. 4).
For every cell shape the library implements (cx in {4, 8, 16, 32}, cy in
{4, 8, 16}) the GPU lattice must equal the oracle's DTrDT replay (O2) bit for
bit after every MCS, with equal net flips and roughness sums, on the same
configuration matrix as the 4x4 parity tests (test_gpu_parity.py)."""
import numpy as np
import pytest

from test_gpu_parity import CONFIGS, _assert_same

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8), (16, 8), (16, 16), (8, 4), (4, 8), (16, 4), (8, 16), (32, 4), (32, 8), (32, 16), (4, 16)]


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def _cases():
    for cx, cy in SHAPES:
        for c in CONFIGS:
            yield pytest.param(cx, cy, c, id="TC{}x{}_L{L}_p{p}_q{q}_B{Bx}x{By}".format(cx, cy, **c))


@pytest.mark.parametrize("cx,cy,c", list(_cases()))
def test_cells_bit_exact(g, oracle, cx, cy, c):
    prm = oracle.Params(L=c["L"], p=c["p"], q=c["q"], seed=c["seed"], Bx=c["Bx"], By=c["By"], cx=cx, cy=cy)
    assert oracle.check_params(prm)
    X, Y = oracle.flat(c["L"])
    with g.Simulation(c["L"], c["p"], c["q"], c["seed"], Bx=c["Bx"], By=c["By"], cx=cx, cy=cy) as sim:
        assert (sim.cx, sim.cy) == (cx, cy)
        net = 0
        for t in range(min(c["n"], 4)):
            net += oracle.dtrdt_run(X, Y, prm, t, 1)[0]
            sim.run(1)
            _assert_same(oracle, sim, X, Y, net, f"TC {cx}x{cy} t={t + 1}")


def test_cells_kpz_256_through_40_mcs(g, oracle):
    """The paper's smallest cell, TC=1,1 (8x8 sites), at L = 256, p = 1, q = 0,
    64 x 64 sub-tiles, compared at log-spaced times up to 40 MCS."""
    prm = oracle.Params(L=256, p=1.0, q=0.0, seed=1, Bx=64, By=64, cx=8, cy=8)
    X, Y = oracle.flat(256)
    net, t = 0, 0
    with g.Simulation(256, 1.0, 0.0, 1, Bx=64, By=64, cx=8, cy=8) as sim:
        for tt in (1, 2, 5, 10, 20, 40):
            net += oracle.dtrdt_run(X, Y, prm, t, tt - t)[0]
            sim.run(tt - t)
            t = tt
            _assert_same(oracle, sim, X, Y, net, f"t={t}")


def test_unsupported_cells_are_refused(g):
    from paper_1705_01022_gb300 import _lib
    for kw in (dict(cx=64, cy=8), dict(cx=8, cy=32), dict(cx=2, cy=2), dict(cx=8, cy=8, scheme=1),
               dict(cx=16, cy=16, scheme=2)):
        with pytest.raises(_lib.OctError):
            g.Simulation(512, 0.5, 0.5, 1, Bx=64, By=64, **kw)
