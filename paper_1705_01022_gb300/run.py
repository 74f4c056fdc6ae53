"""Production runs: roughness at log-spaced times, two-time autocorrelations
and effective exponents (Sec. 2: W of Eq. (3), C of Eq. (5), Eq. (8)).

A run starts from the flat state and advances whole MCS on the GPU. At each
measurement time it takes the exact W^2 (integer S1, S2). With waiting times
given, it snapshots the lattice at the first of them that has been reached
and from then on measures C_h(t, s) and C_s(t, s) at every later measurement
time (one snapshot at a time: a later waiting time replaces the earlier one).

Measurement times follow t_i = max(t_{i-1} + 1, round(t_max^(i/(n-1)))),
i = 0..n-1, after t = 0; waiting times are added to that list.

Effective exponents take Eq. (8) on consecutive pairs (t_j < t_i):
e = (ln E(t_i) - ln E(t_j)) / (ln t_i - ln t_j). The paper prints the time
of the estimate as (t_i - t_j)/2, which for a midpoint must be read as
(t_i + t_j)/2; each estimate also carries the geometric midpoint
sqrt(t_i t_j), the natural one on a log axis.

An ensemble (`ensemble_run`, `--seeds N`) advances N independent
realizations together (DTrDT as one batch, the other block layers as one
handle per realization, each on its own stream) and reports the mean W^2
(and, after a waiting time, the mean C_h and C_s) with standard errors; the
effective exponents of the mean carry jackknife errors over the
realizations.

Command line:
    python -m paper_1705_01022_gb300.run --L 131072 --p 0.95 --q 0.05 \
        --t-max 10000 --points 40 [--wait 100] [--scheme dt|db|dtr] [--seeds N] [--out f.jsonl]
prints one JSON line per measurement, then one summary line.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

SCHEMES = {"dt": 0, "db": 1, "dtr": 2}


def measurement_times(t_max: int, n: int, waits=()) -> list[int]:
    """0, then n log-spaced times ending at t_max (strictly increasing), with the waiting times merged in."""
    if t_max < 1 or n < 1:
        raise ValueError("t_max and n must be >= 1")
    ts = [0]
    for i in range(n):
        t = t_max if n == 1 else int(round(t_max ** (i / (n - 1))))
        t = max(ts[-1] + 1, t)
        if t > t_max:
            break
        ts.append(t)
    if ts[-1] != t_max:
        ts.append(t_max)
    for s in waits:
        if not 0 <= int(s) <= t_max:
            raise ValueError(f"waiting time {s} outside [0, {t_max}]")
    return sorted(set(ts) | {int(s) for s in waits})


def effective_exponents(ts, E, power: float = 1.0) -> list[dict]:
    """Eq. (8) on consecutive pairs of (t, E) with t > 0 and E > 0; `power`
    rescales the exponent (0.5 turns W^2 into W)."""
    pts = [(float(t), float(e)) for t, e in zip(ts, E) if t > 0 and e > 0]
    out = []
    for (tj, ej), (ti, ei) in zip(pts, pts[1:]):
        out.append({"t_j": tj, "t_i": ti, "t_mid": 0.5 * (ti + tj), "t_geo": math.sqrt(ti * tj),
                    "exponent": power * (math.log(ei) - math.log(ej)) / (math.log(ti) - math.log(tj))})
    return out


def production_run(L: int, p: float, q: float, seed: int, t_max: int, points: int, waits=(),
                   scheme: str = "dt", Bx: int = 0, By: int = 0, stream=None, callback=None) -> dict:
    """Runs to t_max and returns {records, beta_eff, wall_s, attempts_per_ns}.

    records: one dict per measurement time (t, w2, s1, s2, net_flips and, after
    a snapshot, s, c_h, c_s). beta_eff: Eq. (8) on W = sqrt(W^2).
    attempts_per_ns: L^2 t_max attempts over the wall time of the whole run,
    measurements included."""
    from . import Simulation
    ts = measurement_times(t_max, points, waits)
    waits = sorted(int(s) for s in waits)
    records = []
    t0 = time.perf_counter()
    with Simulation(L, p, q, seed, Bx=Bx, By=By, scheme=SCHEMES[scheme], stream=stream) as sim:
        t = 0
        for tt in ts:
            sim.run(tt - t)
            t = tt
            m = sim.measure()
            rec = {"t": t, "w2": m.w2, "s1": m.s1, "s2": m.s2, "net_flips": m.net_flips}
            if t in waits:
                sim.snapshot()
            if waits and t > waits[0]:
                ac = sim.measure_ac()
                rec.update({"s": ac.s, "c_h": ac.c_h, "c_s": ac.c_s})
            records.append(rec)
            if callback:
                callback(rec)
        sim.sync()
    wall = time.perf_counter() - t0
    beta = effective_exponents([r["t"] for r in records], [r["w2"] for r in records], power=0.5)
    return {"records": records, "beta_eff": beta, "wall_s": wall,
            "attempts_per_ns": L * L * t_max / (wall * 1e9)}


def jackknife(values, estimator):
    """Jackknife means and standard errors of a vector-valued estimator(samples)
    over the leave-one-out subsets of the sample list (n >= 2); a scalar
    estimator gives one-element lists."""
    n = len(values)
    if n < 2:
        raise ValueError("the jackknife needs at least two samples")
    est = [estimator(values[:i] + values[i + 1:]) for i in range(n)]
    est = [list(e) if isinstance(e, (list, tuple)) else [e] for e in est]
    means = [sum(col) / n for col in zip(*est)]
    errs = [math.sqrt((n - 1) / n * sum((x - m) ** 2 for x in col)) for col, m in zip(zip(*est), means)]
    return means, errs


def _mean_se(x):
    m = sum(x) / len(x)
    return m, math.sqrt(sum((v - m) ** 2 for v in x) / (len(x) - 1) / len(x))


class _Handles:
    """Realizations of a block layer the batched kernel does not run (DTrDB,
    DTrDTr): one simulation handle each, every handle on its own stream, so
    that the device steps of different realizations overlap on the GPU. Same
    interface as the parts of Batch that ensemble_run uses."""

    def __init__(self, L, p, q, seeds, scheme, Bx, By):
        from . import Simulation
        self.sims = []
        try:
            for sd in seeds:
                self.sims.append(Simulation(L, p, q, sd, Bx=Bx, By=By, scheme=SCHEMES[scheme]))
        except Exception:
            self.close()
            raise

    def run(self, n):
        for sim in self.sims:  # asynchronous: every handle enqueues on its own stream
            sim.run(n)

    def measure(self):
        return [sim.measure() for sim in self.sims]

    def snapshot(self, r):
        self.sims[r].snapshot()

    def measure_ac(self, r):
        return self.sims[r].measure_ac()

    def sync(self):
        for sim in self.sims:
            sim.sync()

    def close(self):
        for sim in self.sims:
            sim.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def ensemble_run(L: int, p: float, q: float, seeds, t_max: int, points: int, Bx: int = 0, By: int = 0,
                 stream=None, callback=None, wait: int | None = None, scheme: str = "dt") -> dict:
    """Independent realizations (one per seed) advanced together: DTrDT as one
    batch, DTrDB and DTrDTr as one handle per realization on its own stream;
    returns {records, beta_eff, wall_s, attempts_per_ns}.

    records: per measurement time, t, the mean W^2 over the realizations, its
    standard error and every realization's W^2; with a waiting time s
    (`wait`), every realization is snapshot at s and the records after it
    add the mean C_h(t,s) and C_s(t,s) with their standard errors and every
    realization's C_h. beta_eff: Eq. (8) on W = sqrt(mean W^2) for
    consecutive times, with a jackknife error over the realizations."""
    from . import Batch
    seeds = [int(x) for x in seeds]
    if len(seeds) < 2:
        raise ValueError("an ensemble needs at least two seeds")
    ts = measurement_times(t_max, points, () if wait is None else (wait,))
    shape = (Bx, By) if Bx and By else ()
    records = []
    t0 = time.perf_counter()
    if scheme not in SCHEMES:
        raise ValueError(f"unknown scheme {scheme!r}")
    group = (Batch([(L, p, q, sd) + shape for sd in seeds], stream=stream) if scheme == "dt"
             else _Handles(L, p, q, seeds, scheme, Bx, By))
    with group as b:
        t = 0
        for tt in ts:
            b.run(tt - t)
            t = tt
            ms = b.measure()
            w = [m.w2 for m in ms]
            mean, se = _mean_se(w)
            rec = {"t": t, "w2_mean": mean, "w2_se": se, "w2": w}
            if wait is not None and t == wait:
                for r in range(len(seeds)):
                    b.snapshot(r)
            if wait is not None and t > wait:
                acs = [b.measure_ac(r) for r in range(len(seeds))]
                ch, cs = [a.c_h for a in acs], [a.c_s for a in acs]
                rec["s"] = wait
                rec["c_h_mean"], rec["c_h_se"] = _mean_se(ch)
                rec["c_s_mean"], rec["c_s_se"] = _mean_se(cs)
                rec["c_h"] = ch
            records.append(rec)
            if callback:
                callback(rec)
        b.sync()
    wall = time.perf_counter() - t0
    times = [r["t"] for r in records]
    per_seed = [[r["w2"][i] for r in records] for i in range(len(seeds))]

    def beta_of(samples):
        mean = [sum(col) / len(col) for col in zip(*samples)]
        return [e["exponent"] for e in effective_exponents(times, mean, power=0.5)]

    central = effective_exponents(times, [r["w2_mean"] for r in records], power=0.5)
    _, errs = jackknife(per_seed, beta_of)
    for e, err in zip(central, errs):
        e["error"] = err
    return {"records": records, "beta_eff": central, "wall_s": wall,
            "attempts_per_ns": len(seeds) * L * L * t_max / (wall * 1e9)}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--L", type=int, default=4096)
    ap.add_argument("--p", type=float, default=1.0)
    ap.add_argument("--q", type=float, default=0.0)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--t-max", type=int, default=1000)
    ap.add_argument("--points", type=int, default=30)
    ap.add_argument("--wait", type=int, action="append", default=[], help="waiting time s (repeatable)")
    ap.add_argument("--scheme", choices=sorted(SCHEMES), default="dt")
    ap.add_argument("--Bx", type=int, default=0)
    ap.add_argument("--By", type=int, default=0)
    ap.add_argument("--out", default=None, help="also write the JSON lines to this file")
    ap.add_argument("--seeds", type=int, default=1,
                    help="realizations; with 2 or more, an ensemble (DTrDT as one batch, DTrDB/DTrDTr as concurrent "
                         "handles) whose replica seeds derive from --seed; the first --wait is its waiting time")
    a = ap.parse_args(argv)
    fp = open(a.out, "w") if a.out else None

    def emit(obj):
        line = json.dumps(obj)
        print(line, flush=True)
        if fp:
            fp.write(line + "\n")
            fp.flush()

    if a.seeds >= 2:
        from . import _lib
        seeds = [_lib.oct_replica_seed(a.seed, r) for r in range(a.seeds)]
        res = ensemble_run(a.L, a.p, a.q, seeds, a.t_max, a.points, a.Bx, a.By, callback=emit,
                           wait=a.wait[0] if a.wait else None, scheme=a.scheme)
    else:
        res = production_run(a.L, a.p, a.q, a.seed, a.t_max, a.points, a.wait, a.scheme, a.Bx, a.By,
                             callback=emit)
    emit({"summary": {"L": a.L, "p": a.p, "q": a.q, "seed": a.seed, "seeds": a.seeds, "t_max": a.t_max,
                      "scheme": a.scheme,
                      "wall_s": round(res["wall_s"], 3), "attempts_per_ns": round(res["attempts_per_ns"], 1),
                      "beta_eff": [{k: round(v, 5) for k, v in b.items()} for b in res["beta_eff"]]}})
    if fp:
        fp.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
