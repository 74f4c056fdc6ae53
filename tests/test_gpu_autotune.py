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


def test_tuned_cell_trades_speed_for_fidelity_and_is_bit_exact(g, oracle, tmp_path):
    """The cell tuner measures every supported cell's rate and its W^2 against
    the coarsest cell, picks the fastest within the allowed shift, records it,
    and the run on the chosen cell is the oracle's DTrDT with that cell."""
    from paper_1705_01022_gb300 import autotune as at
    L, p, q, seed, Bx, By = 1024, 0.95, 0.05, 4, 64, 64
    cache = at.TuneCache.load(str(tmp_path / "tune.json"))
    rec = at.choose_cell(L, p, q, Bx, By, max_shift=0.01, cache=cache)
    assert len(rec["table"]) == len(at.CELLS) and rec["reference"] == [32, 16]
    rows = {(r["cx"], r["cy"]): r for r in rec["table"]}
    assert all(r["attempts_per_ns"] > 0 for r in rec["table"])
    # finer cells are faster, and 4x4 cells lower W^2 well below the coarse cells (Sec. 4.2)
    assert rows[(4, 4)]["attempts_per_ns"] > 2 * rows[(16, 16)]["attempts_per_ns"]
    assert all(x < 0.99 for x in rows[(4, 4)]["w2_ratio"]), rows[(4, 4)]
    chosen = rows[(rec["cx"], rec["cy"])]
    assert all(abs(x - 1) <= 0.01 for x in chosen["w2_ratio"])
    ok = [r for r in rec["table"] if all(abs(x - 1) <= 0.01 for x in r["w2_ratio"])]
    assert chosen["attempts_per_ns"] == max(r["attempts_per_ns"] for r in ok)
    again = at.choose_cell(L, p, q, Bx, By, max_shift=0.01, cache=at.TuneCache.load(cache.path))
    assert again["when"] == rec["when"]
    # with no shift allowed only the reference qualifies
    assert (at.pick_cell(rec["table"], 0.0)["cx"], at.pick_cell(rec["table"], 0.0)["cy"]) == (32, 16)
    prm = oracle.Params(L=L, p=p, q=q, seed=seed, Bx=Bx, By=By, cx=rec["cx"], cy=rec["cy"])
    X, Y = oracle.flat(L)
    net = oracle.dtrdt_run(X, Y, prm, 0, 2)[0]
    with g.Simulation(L, p, q, seed, Bx=Bx, By=By, cx=rec["cx"], cy=rec["cy"]) as sim:
        sim.run(2)
        Xg, Yg = oracle.unpack_canonical(sim.lattice(), L)
        m = sim.measure()
    assert np.array_equal(Xg, X) and np.array_equal(Yg, Y)
    assert m.net_flips == net
