"""The block-tile autotuner on the GPU: it measures every shape, records its
choice, and the tuned simulation is the DTrDT dynamics of that shape, bit for
bit against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def test_tuned_shape_is_recorded_and_bit_exact(g, oracle, tmp_path):
    from paper_1705_01022_gb300 import autotune as at
    L, p, q, seed = 2048, 0.95, 0.05, 9
    cache = at.TuneCache.load(str(tmp_path / "tune.json"))
    sim = at.tuned_simulation(L, p, q, seed, cache=cache, mcs=1)
    rec = sim.tuning
    assert (rec["Bx"], rec["By"]) in at.candidates(L)
    assert len(rec["table"]) == len(at.candidates(L))
    assert all(r["attempts_per_ns"] > 0 for r in rec["table"])
    assert rec["attempts_per_ns"] == max(r["attempts_per_ns"] for r in rec["table"])
    # the recorded choice is reused without measuring again
    again = at.choose(L, p, q, cache=at.TuneCache.load(cache.path))
    assert (again["Bx"], again["By"]) == (rec["Bx"], rec["By"]) and again["when"] == rec["when"]
    # and the run on it is the oracle's DTrDT with that sub-tile
    prm = oracle.Params(L=L, p=p, q=q, seed=seed, Bx=rec["Bx"], By=rec["By"])
    X, Y = oracle.flat(L)
    net = oracle.dtrdt_run(X, Y, prm, 0, 3)[0]
    with sim:
        sim.run(3)
        Xg, Yg = oracle.unpack_canonical(sim.lattice(), L)
        m = sim.measure()
    assert np.array_equal(Xg, X) and np.array_equal(Yg, Y)
    assert m.net_flips == net
