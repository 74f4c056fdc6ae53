"""Production runs on the GPU (W^2 at log-spaced times and the two-time
autocorrelations after a waiting time, Sec. 2) against the oracle's replay of
the same schedule: every record's W^2, C_h and C_s are the same doubles
(they come from equal integer sums)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


@pytest.mark.parametrize("scheme,L,Bx,By,p,q", [
    ("dt", 256, 64, 64, 0.95, 0.05),
    ("dt", 512, 128, 32, 1.0, 0.0),
    ("db", 256, 64, 64, 0.95, 0.05),
    ("dtr", 256, 64, 64, 0.5, 0.5),
])
def test_production_run_matches_oracle(g, oracle, scheme, L, Bx, By, p, q):
    from oracle import Params, SCHEME_DB, SCHEME_DT, SCHEME_DTR
    from paper_1705_01022_gb300 import run as prun
    res = prun.production_run(L, p, q, 9, t_max=24, points=6, waits=[5], scheme=scheme, Bx=Bx, By=By)
    prm = Params(L=L, p=p, q=q, seed=9, Bx=Bx, By=By,
                 scheme={"dt": SCHEME_DT, "db": SCHEME_DB, "dtr": SCHEME_DTR}[scheme])
    X, Y = oracle.flat(L)
    t, net, snap = 0, 0, None
    for r in res["records"]:
        net += oracle.dtrdt_run(X, Y, prm, t, r["t"] - t)[0]
        t = r["t"]
        s1, s2, _ = oracle.w2_sums(X, Y)
        assert (r["s1"], r["s2"], r["net_flips"]) == (s1, s2, net), t
        assert r["w2"] == oracle.w2(X, Y), t
        if t == 5:
            snap = (X.copy(), Y.copy())
        if t > 5:
            a = oracle.two_time(X, Y, *snap)
            assert (r["s"], r["c_h"], r["c_s"]) == (5, a["c_h"], a["c_s"]), t
    assert [r["t"] for r in res["records"]][-1] == 24


@pytest.mark.parametrize("L,p,q,Bx,By", [(256, 1.0, 0.0, 64, 64), (320, 0.5, 0.5, 32, 32)])
def test_ensemble_run_matches_plain_runs(g, L, p, q, Bx, By):
    """Every realization of the batched ensemble has the W^2 of the same seed
    run alone, at every measurement time."""
    from paper_1705_01022_gb300 import run as prun
    seeds = [g._lib.oct_replica_seed(7, r) for r in range(5)]
    res = prun.ensemble_run(L, p, q, seeds, t_max=30, points=8, Bx=Bx, By=By)
    for i, sd in enumerate(seeds):
        with g.Simulation(L, p, q, sd, Bx=Bx, By=By) as sim:
            t = 0
            for r in res["records"]:
                sim.run(r["t"] - t)
                t = r["t"]
                assert r["w2"][i] == sim.measure().w2, (i, t)
    assert all(b["error"] > 0 for b in res["beta_eff"])


def test_ensemble_autocorrelations_match_plain_runs(g):
    """The batch's per-replica snapshot and C_h, C_s equal those of the same
    seed run alone (exact doubles from equal integer sums)."""
    from paper_1705_01022_gb300 import run as prun
    L, p, q, Bx, By, s = 256, 0.95, 0.05, 64, 64, 4
    seeds = [g._lib.oct_replica_seed(9, r) for r in range(4)]
    res = prun.ensemble_run(L, p, q, seeds, t_max=20, points=6, Bx=Bx, By=By, wait=s)
    for i, sd in enumerate(seeds):
        with g.Simulation(L, p, q, sd, Bx=Bx, By=By) as sim:
            t = 0
            for r in res["records"]:
                sim.run(r["t"] - t)
                t = r["t"]
                if t == s:
                    sim.snapshot()
                if t > s:
                    ac = sim.measure_ac()
                    assert r["c_h"][i] == ac.c_h, (i, t)


def test_batch_autocorrelation_errors(g):
    with g.Batch([(128, 1.0, 0.0, 1), (128, 0.5, 0.5, 2)]) as b:
        b.run(2)
        with pytest.raises(g.OctError):
            b.measure_ac(0)  # no snapshot yet
        b.snapshot(1)
        b.run(1)
        ac = b.measure_ac(1)
        assert (ac.t, ac.s) == (3, 2)
        assert 0.0 < ac.c_s < 0.25
        with pytest.raises(g.OctError):
            b.measure_ac(5)  # no such slot


@pytest.mark.parametrize("scheme,sch", [("db", 1), ("dtr", 2)])
def test_ensemble_of_other_block_layers_on_concurrent_streams(g, scheme, sch):
    """DTrDB / DTrDTr ensembles (one handle per realization, interleaved on
    their own streams) equal the same seeds run one after another."""
    from paper_1705_01022_gb300 import run as prun
    L, p, q, Bx, By, s = 256, 0.95, 0.05, 64, 64, 3
    seeds = [101, 202, 303]
    res = prun.ensemble_run(L, p, q, seeds, t_max=12, points=5, Bx=Bx, By=By, wait=s, scheme=scheme)
    for i, sd in enumerate(seeds):
        with g.Simulation(L, p, q, sd, Bx=Bx, By=By, scheme=sch) as sim:
            t = 0
            for r in res["records"]:
                sim.run(r["t"] - t)
                t = r["t"]
                assert r["w2"][i] == sim.measure().w2, (i, t)
                if t == s:
                    sim.snapshot()
                if t > s:
                    assert r["c_h"][i] == sim.measure_ac().c_h, (i, t)


def test_waiting_time_zero(g, oracle):
    """s = 0: the snapshot is the flat start itself (C_h(0,0) = W^2(0) = 1/4);
    later C_h(t,0), C_s(t,0) equal the oracle's, alone and in an ensemble."""
    from oracle import Params
    from paper_1705_01022_gb300 import run as prun
    L, p, q = 256, 1.0, 0.0
    res = prun.production_run(L, p, q, 5, t_max=6, points=4, waits=[0], Bx=64, By=64)
    X, Y = oracle.flat(L)
    Xs, Ys = X.copy(), Y.copy()
    t = 0
    for r in res["records"]:
        oracle.dtrdt_run(X, Y, Params(L=L, p=p, q=q, seed=5, Bx=64, By=64), t, r["t"] - t)
        t = r["t"]
        if t > 0:
            a = oracle.two_time(X, Y, Xs, Ys)
            assert (r["s"], r["c_h"], r["c_s"]) == (0, a["c_h"], a["c_s"]), t
    assert res["records"][0]["w2"] == 0.25
    seeds = [g._lib.oct_replica_seed(3, r) for r in range(3)]
    ens = prun.ensemble_run(L, p, q, seeds, t_max=6, points=4, Bx=64, By=64, wait=0)
    for i, sd in enumerate(seeds):
        X, Y = oracle.flat(L)
        t = 0
        for r in ens["records"]:
            oracle.dtrdt_run(X, Y, Params(L=L, p=p, q=q, seed=sd, Bx=64, By=64), t, r["t"] - t)
            t = r["t"]
            if t > 0:
                assert r["c_h"][i] == oracle.two_time(X, Y, Xs, Ys)["c_h"], (i, t)
