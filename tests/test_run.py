"""Host logic of production runs (Sec. 2: W of Eq. (3), C of Eq. (5),
effective exponents of Eq. (8)), on CPU.

* Measurement times: t = 0, then the log-spaced schedule, strictly
  increasing, ending at t_max, with the waiting times merged in.
* Eq. (8): a pure power law E = c t^e gives e on every pair, whatever c;
  power 0.5 turns the exponent of W^2 into that of W; t <= 0 and E <= 0 are
  skipped (ln undefined).
* production_run's bookkeeping (when it snapshots, which records carry C)
  with the simulation replaced by an oracle-backed stand-in: every record
  equals the oracle's own W^2 and two-time values at that time.
* Ensembles: the jackknife error of a sample mean is the classical standard
  error (an identity); ensemble_run's per-realization W^2 equal the oracle's,
  the mean and its error follow, and the exponent errors shrink with more
  realizations.
"""
import math

import numpy as np
import pytest

from paper_1705_01022_gb300 import run as prun


def test_measurement_times_schedule():
    ts = prun.measurement_times(10_000, 40)
    assert ts[0] == 0 and ts[-1] == 10_000
    assert all(b > a for a, b in zip(ts, ts[1:]))
    assert len(ts) == 41
    # the first log-spaced times collide at small t and are pushed up by one
    assert ts[1:6] == [1, 2, 3, 4, 5]
    # later ones follow round(t_max^(i/(n-1)))
    assert ts[30] == round(10_000 ** (29 / 39))
    ts2 = prun.measurement_times(100, 5, waits=[7, 100, 0])
    assert ts2 == sorted(set(ts2)) and {0, 7, 100} <= set(ts2)
    assert prun.measurement_times(5, 1) == [0, 5]
    with pytest.raises(ValueError):
        prun.measurement_times(100, 5, waits=[101])
    with pytest.raises(ValueError):
        prun.measurement_times(0, 5)


@pytest.mark.parametrize("c,e", [(1.0, 0.2414), (0.37, 0.5), (12.5, -1.3)])
def test_effective_exponent_of_a_power_law(c, e):
    ts = [0, 1, 3, 10, 31, 100, 316, 1000]
    E = [c * t ** e if t > 0 else 0.0 for t in ts]
    out = prun.effective_exponents(ts, E)
    assert len(out) == len(ts) - 2  # t = 0 dropped
    for r in out:
        assert r["exponent"] == pytest.approx(e, rel=1e-12, abs=1e-12)
        assert r["t_j"] < r["t_i"]
        assert r["t_mid"] == 0.5 * (r["t_i"] + r["t_j"])
        assert r["t_geo"] == pytest.approx(math.sqrt(r["t_i"] * r["t_j"]))
    w = prun.effective_exponents(ts, [x ** 2 for x in E], power=0.5)
    for r in w:
        assert r["exponent"] == pytest.approx(e, rel=1e-12, abs=1e-12)


def test_effective_exponent_skips_nonpositive_values():
    out = prun.effective_exponents([1, 2, 4, 8], [1.0, -1.0, 4.0, 8.0])
    assert [(r["t_j"], r["t_i"]) for r in out] == [(1.0, 4.0), (4.0, 8.0)]
    assert out[0]["exponent"] == pytest.approx(1.0)


class _OracleSim:
    """Stand-in for the GPU Simulation: the oracle's DTrDT replay."""

    def __init__(self, oracle, L, p, q, seed, Bx=0, By=0, scheme=0, stream=None):
        from oracle import Params, SCHEME_DB, SCHEME_DT, SCHEME_DTR
        self.o = oracle
        self.prm = Params(L=L, p=p, q=q, seed=seed, Bx=Bx or 32, By=By or 32,
                          scheme={0: SCHEME_DT, 1: SCHEME_DB, 2: SCHEME_DTR}[scheme])
        self.X, self.Y = oracle.flat(L)
        self.t, self.net, self.snap = 0, 0, None

    def run(self, n):
        self.net += self.o.dtrdt_run(self.X, self.Y, self.prm, self.t, n)[0]
        self.t += n

    def measure(self):
        s1, s2, _ = self.o.w2_sums(self.X, self.Y)
        return type("W", (), dict(w2=self.o.w2(self.X, self.Y), s1=s1, s2=s2, net_flips=self.net))

    def snapshot(self):
        self.snap = (self.X.copy(), self.Y.copy(), self.t)

    def measure_ac(self):
        if self.snap is None:
            raise RuntimeError("no snapshot")
        a = self.o.two_time(self.X, self.Y, self.snap[0], self.snap[1])
        return type("A", (), dict(s=self.snap[2], c_h=a["c_h"], c_s=a["c_s"]))

    def sync(self):
        pass

    def close(self):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        pass


@pytest.mark.parametrize("scheme", ["dt", "db", "dtr"])
def test_production_run_bookkeeping(oracle, monkeypatch, scheme):
    import paper_1705_01022_gb300 as pkg
    from oracle import Params, SCHEME_DB, SCHEME_DT, SCHEME_DTR
    monkeypatch.setattr(pkg, "Simulation", lambda *a, **k: _OracleSim(oracle, *a, **k))
    L, p, q, seed = 64, 0.95, 0.05, 5
    seen = []
    res = prun.production_run(L, p, q, seed, t_max=12, points=5, waits=[3], scheme=scheme,
                              callback=seen.append)
    recs = res["records"]
    assert seen == recs
    assert [r["t"] for r in recs] == prun.measurement_times(12, 5, [3])
    # replay independently and compare every record
    prm = Params(L=L, p=p, q=q, seed=seed, Bx=32, By=32,
                 scheme={"dt": SCHEME_DT, "db": SCHEME_DB, "dtr": SCHEME_DTR}[scheme])
    X, Y = oracle.flat(L)
    t, snap = 0, None
    for r in recs:
        oracle.dtrdt_run(X, Y, prm, t, r["t"] - t)
        t = r["t"]
        assert r["w2"] == oracle.w2(X, Y)
        if t == 3:
            snap = (X.copy(), Y.copy())
        if t > 3:
            a = oracle.two_time(X, Y, *snap)
            assert (r["s"], r["c_h"], r["c_s"]) == (3, a["c_h"], a["c_s"])
        else:
            assert "c_h" not in r
    assert recs[0]["w2"] == 0.25  # flat start
    assert len(res["beta_eff"]) == len(recs) - 2


def test_jackknife_of_the_mean_is_the_standard_error():
    rng = np.random.default_rng(4)
    x = rng.normal(size=13).tolist()
    (m,), (e,) = prun.jackknife(x, lambda v: sum(v) / len(v))
    assert m == pytest.approx(np.mean(x), rel=1e-12)
    assert e == pytest.approx(np.std(x, ddof=1) / np.sqrt(len(x)), rel=1e-10)
    with pytest.raises(ValueError):
        prun.jackknife([1.0], lambda v: v[0])


class _OracleBatch:
    """Stand-in for the GPU Batch: one oracle replay per replica."""

    def __init__(self, oracle, replicas, stream=None):
        from oracle import Params
        self.o = oracle
        self.reps = []
        for L, p, q, seed, Bx, By in replicas:
            X, Y = oracle.flat(L)
            self.reps.append([Params(L=L, p=p, q=q, seed=seed, Bx=Bx, By=By), X, Y])
        self.t = 0

    def run(self, n):
        for prm, X, Y in self.reps:
            self.o.dtrdt_run(X, Y, prm, self.t, n)
        self.t += n

    def measure(self):
        return [type("W", (), dict(w2=self.o.w2(X, Y))) for _, X, Y in self.reps]

    def snapshot(self, r):
        _, X, Y = self.reps[r]
        self.snaps = getattr(self, "snaps", {})
        self.snaps[r] = (X.copy(), Y.copy())

    def measure_ac(self, r):
        _, X, Y = self.reps[r]
        a = self.o.two_time(X, Y, *self.snaps[r])
        return type("A", (), dict(c_h=a["c_h"], c_s=a["c_s"]))

    def sync(self):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        pass


def test_ensemble_run_bookkeeping(oracle, monkeypatch):
    import paper_1705_01022_gb300 as pkg
    from oracle import Params
    monkeypatch.setattr(pkg, "Batch", lambda reps, stream=None: _OracleBatch(oracle, reps))
    L, p, q, seeds = 64, 1.0, 0.0, [11, 12, 13, 14]
    res = prun.ensemble_run(L, p, q, seeds, t_max=10, points=4, Bx=32, By=32)
    recs = res["records"]
    assert [r["t"] for r in recs] == prun.measurement_times(10, 4)
    for i, sd in enumerate(seeds):
        X, Y = oracle.flat(L)
        t = 0
        for r in recs:
            oracle.dtrdt_run(X, Y, Params(L=L, p=p, q=q, seed=sd, Bx=32, By=32), t, r["t"] - t)
            t = r["t"]
            assert r["w2"][i] == oracle.w2(X, Y)
    for r in recs:
        assert r["w2_mean"] == pytest.approx(np.mean(r["w2"]), rel=1e-14)
        assert r["w2_se"] == pytest.approx(np.std(r["w2"], ddof=1) / 2, rel=1e-12)
    assert recs[0]["w2_se"] == 0.0  # every realization starts flat
    assert all(b["error"] > 0 for b in res["beta_eff"])
    with pytest.raises(ValueError):
        prun.ensemble_run(L, p, q, [1], t_max=10, points=4)


def test_ensemble_run_with_waiting_time(oracle, monkeypatch):
    import paper_1705_01022_gb300 as pkg
    from oracle import Params
    monkeypatch.setattr(pkg, "Batch", lambda reps, stream=None: _OracleBatch(oracle, reps))
    L, p, q, seeds, s = 64, 0.95, 0.05, [21, 22, 23], 3
    res = prun.ensemble_run(L, p, q, seeds, t_max=12, points=4, Bx=32, By=32, wait=s)
    recs = res["records"]
    assert s in [r["t"] for r in recs]
    for r in recs:
        assert ("c_h_mean" in r) == (r["t"] > s)
    # every realization's C_h against the oracle's own replay
    for i, sd in enumerate(seeds):
        X, Y = oracle.flat(L)
        t, snap = 0, None
        for r in recs:
            oracle.dtrdt_run(X, Y, Params(L=L, p=p, q=q, seed=sd, Bx=32, By=32), t, r["t"] - t)
            t = r["t"]
            if t == s:
                snap = (X.copy(), Y.copy())
            if t > s:
                assert r["c_h"][i] == oracle.two_time(X, Y, *snap)["c_h"]
    for r in recs:
        if r["t"] > s:
            assert r["c_h_mean"] == pytest.approx(np.mean(r["c_h"]), rel=1e-14)
            assert r["c_h_se"] == pytest.approx(np.std(r["c_h"], ddof=1) / np.sqrt(3), rel=1e-10)


def test_command_line(oracle, monkeypatch, tmp_path, capsys):
    """`python -m paper_1705_01022_gb300.run`: one JSON line per measurement
    time, then a summary; the same lines go to --out."""
    import json

    import paper_1705_01022_gb300 as pkg
    monkeypatch.setattr(pkg, "Simulation", lambda *a, **k: _OracleSim(oracle, *a, **k))
    out = tmp_path / "run.jsonl"
    rc = prun.main(["--L", "64", "--p", "0.95", "--q", "0.05", "--t-max", "8", "--points", "4",
                    "--wait", "2", "--Bx", "32", "--By", "32", "--out", str(out)])
    assert rc == 0
    lines = [json.loads(x) for x in capsys.readouterr().out.splitlines()]
    assert lines == [json.loads(x) for x in out.read_text().splitlines()]
    recs, summary = lines[:-1], lines[-1]["summary"]
    assert [r["t"] for r in recs] == prun.measurement_times(8, 4, [2])
    assert summary["L"] == 64 and summary["seeds"] == 1 and len(summary["beta_eff"]) == len(recs) - 2
    assert all("c_h" in r for r in recs if r["t"] > 2)


@pytest.mark.parametrize("scheme", ["db", "dtr"])
def test_ensemble_of_other_block_layers(oracle, monkeypatch, scheme):
    """DTrDB and DTrDTr ensembles run one handle per realization; every
    realization's W^2 and C_h equal the oracle's replay of that seed."""
    import paper_1705_01022_gb300 as pkg
    from oracle import Params, SCHEME_DB, SCHEME_DTR
    monkeypatch.setattr(pkg, "Simulation", lambda *a, **k: _OracleSim(oracle, *a, **k))
    L, p, q, seeds, s = 64, 0.95, 0.05, [31, 32], 2
    res = prun.ensemble_run(L, p, q, seeds, t_max=8, points=4, Bx=32, By=32, wait=s, scheme=scheme)
    osch = {"db": SCHEME_DB, "dtr": SCHEME_DTR}[scheme]
    for i, sd in enumerate(seeds):
        X, Y = oracle.flat(L)
        t, snap = 0, None
        for r in res["records"]:
            oracle.dtrdt_run(X, Y, Params(L=L, p=p, q=q, seed=sd, Bx=32, By=32, scheme=osch), t, r["t"] - t)
            t = r["t"]
            assert r["w2"][i] == oracle.w2(X, Y)
            if t == s:
                snap = (X.copy(), Y.copy())
            if t > s:
                assert r["c_h"][i] == oracle.two_time(X, Y, *snap)["c_h"]
    with pytest.raises(ValueError):
        prun.ensemble_run(L, p, q, seeds, t_max=8, points=4, scheme="cdb")
