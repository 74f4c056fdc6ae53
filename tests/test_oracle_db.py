"""Pins for the DTrDB replay: DTr at device level, single-hit dead border (DB)
at block level (Sec. 3.1, block layer; the scheme the paper ends up
recommending, Sec. 5).

* every thread cell makes exactly cx*cy attempts per MCS, at sites uniform
  over its whole cell (no domain sets);
* with only one of p, q non-zero, carrying out the border attempts of a step
  together with the bulk is the same dynamics as delaying them (the paper's
  statement), and no slope bit is ever flipped twice in a step;
* with both non-zero, ignoring the borders lets two accepted flips hit the
  same slope bit and breaks the lattice invariants, while delayed borders
  (bulk, then borders, then corners) keep every phase conflict-free;
* on the 4x4 torus with 2x2 cells DB reduces to the exact master equation of
  a uniformly chosen site per step (the same as DT's degenerate case);
* DB samples the lattice more like true RS than DT at equal cell size."""
import numpy as np
import pytest
from scipy import stats

from oracle import master_eq as me

DB, IGN = 1, 2


@pytest.mark.parametrize("cfg", [dict(L=64, Bx=32, By=32, cx=8, cy=8),
                                 dict(L=128, Bx=32, By=16, cx=4, cy=4),
                                 dict(L=64, Bx=16, By=16, cx=16, cy=8)],
                         ids=lambda c: "L{L}_B{Bx}x{By}_TC{cx}x{cy}".format(**c))
@pytest.mark.parametrize("pq", [(1.0, 0.0), (0.6, 0.3)])
def test_db_schedule_complete_and_conflict_free(oracle, cfg, pq):
    prm = oracle.Params(p=pq[0], q=pq[1], seed=7, scheme=DB, **cfg)
    L, cx, cy = prm.L, prm.cx, prm.cy
    X, Y = oracle.flat(L)
    for t in range(3):
        _, att, conf = oracle.dtrdt_run(X, Y, prm, t, 1, count_attempts=True, check_conflicts=True)
        assert conf == 0
        ox, oy, _ = oracle.mcs_draw(prm, t)
        a = np.roll(att, (-oy, -ox), axis=(0, 1))
        per_tc = a.reshape(L // cy, cy, L // cx, cx).sum(axis=(1, 3))
        assert np.all(per_tc == cx * cy)
        assert oracle.invariants(X, Y) == 0


def test_db_sites_uniform_over_the_cell(oracle):
    prm = oracle.Params(L=128, p=1.0, q=0.0, seed=3, Bx=64, By=32, scheme=DB)
    X, Y = oracle.flat(prm.L)
    pos = np.zeros((4, 4))
    for t in range(30):
        _, att, _ = oracle.dtrdt_run(X, Y, prm, t, 1, count_attempts=True)
        ox, oy, _ = oracle.mcs_draw(prm, t)
        pos += np.roll(att, (-oy, -ox), axis=(0, 1)).reshape(32, 4, 32, 4).sum(axis=(0, 2))
    chi = stats.chisquare(pos.reshape(-1))
    assert chi.pvalue > 1e-4, chi


@pytest.mark.parametrize("pq", [(1.0, 0.0), (0.0, 1.0), (0.7, 0.0), (0.0, 0.4)])
def test_borders_together_equal_delayed_when_one_rate_vanishes(oracle, pq):
    out = []
    for scheme in (DB, IGN):
        X, Y = oracle.flat(64)
        prm = oracle.Params(L=64, p=pq[0], q=pq[1], seed=5, Bx=32, By=32, cx=8, cy=8, scheme=scheme)
        _, _, conf = oracle.dtrdt_run(X, Y, prm, 0, 6, check_conflicts=True)
        assert conf == 0
        out.append((X, Y))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_delayed_borders_are_needed_when_both_rates_are_positive(oracle):
    broken = 0
    for seed in range(6):
        for scheme in (DB, IGN):
            X, Y = oracle.flat(64)
            prm = oracle.Params(L=64, p=0.5, q=0.5, seed=seed, Bx=32, By=32, cx=8, cy=8, scheme=scheme)
            _, _, conf = oracle.dtrdt_run(X, Y, prm, 0, 4, check_conflicts=True)
            if scheme == DB:
                assert conf == 0 and oracle.invariants(X, Y) == 0
            else:
                broken += conf > 0
    assert broken >= 3


def test_db_matches_master_equation(oracle):
    states, index = me.reachable_states()
    pe, qe = oracle.threshold32(0.7) / 2**32, oracle.threshold32(0.2) / 2**32
    pi = me.distribution(me.dtrdt_mcs_matrix(states, index, pe, qe), 1, len(states))
    prm = oracle.Params(L=4, p=0.7, q=0.2, seed=0, Bx=2, By=2, cx=2, cy=2, scheme=DB)
    X, Y = oracle.dtrdt_many(prm, 9000, 200_000, 1)
    counts = np.zeros(len(states))
    for r in range(X.shape[0]):
        counts[index[me.bits_to_code(X[r], Y[r])]] += 1
    assert me.g_test(counts, pi)[2] > 1e-4


def test_db_samples_closer_to_rs_than_dt(oracle):
    L, n, t = 128, 48, 4

    def mean_w2(scheme=None):
        w = []
        for s in range(n):
            X, Y = oracle.flat(L)
            if scheme is None:
                oracle.seq_rs(X, Y, 1.0, 0.0, 1000 + s, 0, t)
            else:
                oracle.dtrdt_run(X, Y, oracle.Params(L=L, p=1.0, q=0.0, seed=2000 + s, Bx=32, By=32,
                                                     scheme=scheme), 0, t)
            w.append(oracle.w2(X, Y))
        return np.mean(w)

    rs, dt, db = mean_w2(), mean_w2(0), mean_w2(DB)
    assert dt / rs < db / rs < 1.0, (dt / rs, db / rs)
