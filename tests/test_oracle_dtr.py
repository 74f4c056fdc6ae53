"""Pins for the oracle's DTrDTr block layer (double tiling whose block-layer
origin moves to a random position after every collective step, Sec. 4.1.2).

* Schedule: conflict-free, one MCS = L^2 attempts, invariants hold, at several
  sub-tile and thread-cell shapes.
* Pattern: in every step the attempts fill one active sub-cell per shifted
  cell: all (lx - c0) mod cx < cx/2 for a common c0, and the shifted cells
  that hold them are all different.  c0 is uniform over [0, cx) (DT only uses
  0 and cx/2).
* The grid the paper attributes to DTrDT: with 4 x 4 cells, DT never attempts
  the sites x = 4i+2 and x = 4i+5 of a row in one step, while it does attempt
  4i+1 and 4i+4 together; under DTrDTr both pairs occur equally often.
* Exact 4 x 4 master equation (B = 2, 2 x 2 cells): a moving origin of one
  cell per sub-tile only relabels the set, so DTrDTr has DTrDT's transition
  matrix; the G-test pins eligibility, acceptance and wrapping of this path.
* Statistics: the W^2 prefactor of DTrDTr is within a few percent of
  DTrDT's (the paper found no substantial improvement).
"""
import numpy as np
import pytest

from oracle import SCHEME_DT, SCHEME_DTR
from oracle import master_eq as me

CONFIGS = [
    dict(L=64, Bx=32, By=16, cx=4, cy=4),
    dict(L=128, Bx=64, By=64, cx=4, cy=4),
    dict(L=128, Bx=32, By=32, cx=8, cy=8),
    dict(L=64, Bx=32, By=32, cx=8, cy=4),
    dict(L=64, Bx=16, By=8, cx=2, cy=2),
    dict(L=512, Bx=256, By=64, cx=4, cy=4),
]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "L{L}_B{Bx}x{By}_TC{cx}x{cy}".format(**c))
def test_dtr_schedule_conflict_free_and_complete(oracle, cfg):
    prm = oracle.Params(p=0.6, q=0.3, seed=5, scheme=SCHEME_DTR, **cfg)
    assert oracle.check_params(prm)
    X, Y = oracle.flat(prm.L)
    for t in range(2):
        net, att, conf = oracle.dtrdt_run(X, Y, prm, t, 1, count_attempts=True, check_conflicts=True)
        assert conf == 0
        assert att.sum() == prm.L ** 2
        assert oracle.invariants(X, Y) == 0


@pytest.mark.parametrize("cfg", CONFIGS[:5], ids=lambda c: "B{Bx}x{By}_TC{cx}x{cy}".format(**c))
def test_dtr_attempts_fill_shifted_cells(oracle, cfg):
    prm = oracle.Params(p=1.0, q=0.0, seed=11, scheme=SCHEME_DTR, **cfg)
    cx, cy, Bx, By = prm.cx, prm.cy, prm.Bx, prm.By
    c0_seen = np.zeros(cx, dtype=int)
    for s in range(cx * cy):
        for T in range(3):
            lx, ly = oracle.subtile_step_sites(prm, 2, 1, T, s)
            # a common phase of the active sub-cell in x and in y
            c0 = [c for c in range(cx) if np.all((lx - c) % cx < cx // 2)]
            r0 = [r for r in range(cy) if np.all((ly - r) % cy < cy // 2)]
            assert c0 and r0
            if len(c0) > 1 or len(r0) > 1:
                continue  # every cell drew the same offset: the phase is ambiguous
            # one attempt per shifted cell
            cell = ((lx - c0[0]) % Bx // cx) + (Bx // cx) * ((ly - r0[0]) % By // cy)
            assert len(set(cell.tolist())) == len(cell)
            c0_seen[c0[0]] += 1
    if cx > 2:
        assert np.all(c0_seen > 0), c0_seen  # the phase takes every value, not only 0 and cx/2


def _pair_counts(oracle, scheme, n_steps=4000):
    """Co-attempts in one step of the sites (x, x+3) of a row, split by x mod 4."""
    prm = oracle.Params(L=128, p=1.0, q=0.0, seed=17, Bx=64, By=64, scheme=scheme)
    counts = np.zeros(4, dtype=int)
    rng = np.random.default_rng(0)
    for _ in range(n_steps):
        t, k, T, s = int(rng.integers(0, 1000)), int(rng.integers(0, 4)), int(rng.integers(0, 4)), int(rng.integers(0, 16))
        lx, ly = oracle.subtile_step_sites(prm, t, k, T, s)
        hit = np.zeros((64, 64 + 3), dtype=bool)
        hit[ly, lx] = True
        both = hit[:, :61] & hit[:, 3:64]
        for a in range(4):
            counts[a] += int(both[:, a::4].sum())
    return counts


def test_dtr_removes_the_double_tiling_grid(oracle):
    dt = _pair_counts(oracle, SCHEME_DT)
    dtr = _pair_counts(oracle, SCHEME_DTR)
    # DT: x = 4i+2 (sub-cell dx = 1) and 4i+5 (dx = 0 of the next cell) never together
    assert dt[2] == 0 and dt[1] > 0
    # DTrDTr: the pattern is translation invariant
    assert np.all(dtr > 0)
    assert dtr.max() / dtr.min() < 1.25, dtr


def test_dtr_matches_master_equation(oracle):
    states, index = me.reachable_states()
    pe, qe = oracle.threshold32(0.7) / 2**32, oracle.threshold32(0.2) / 2**32
    pi = me.distribution(me.dtrdt_mcs_matrix(states, index, pe, qe), 1, len(states))
    prm = oracle.Params(L=4, p=0.7, q=0.2, seed=0, Bx=2, By=2, cx=2, cy=2, scheme=SCHEME_DTR)
    X, Y = oracle.dtrdt_many(prm, 9100, 200_000, 1)
    counts = np.zeros(len(states))
    for r in range(X.shape[0]):
        counts[index[me.bits_to_code(X[r], Y[r])]] += 1
    assert me.g_test(counts, pi)[2] > 1e-4


def test_dtr_symmetry_h_to_minus_h(oracle):
    L = 64
    prm = oracle.Params(L=L, p=0.7, q=0.2, seed=23, Bx=32, By=32, scheme=SCHEME_DTR)
    prm_sw = oracle.Params(L=L, p=0.2, q=0.7, seed=23, Bx=32, By=32, scheme=SCHEME_DTR)
    X, Y = oracle.flat(L)
    Xc, Yc = 1 - X, 1 - Y
    n1 = oracle.dtrdt_run(X, Y, prm, 0, 5)[0]
    n2 = oracle.dtrdt_run(Xc, Yc, prm_sw, 0, 5)[0]
    assert np.array_equal(Xc, 1 - X) and np.array_equal(Yc, 1 - Y)
    assert n2 == -n1


def test_dtr_prefactor_close_to_dt(oracle):
    L, n, t = 128, 48, 4

    def mean_w2(scheme):
        w = []
        for s in range(n):
            X, Y = oracle.flat(L)
            oracle.dtrdt_run(X, Y, oracle.Params(L=L, p=1.0, q=0.0, seed=3000 + s, Bx=32, By=32,
                                                 scheme=scheme), 0, t)
            w.append(oracle.w2(X, Y))
        return np.mean(w)

    dt, dtr = mean_w2(SCHEME_DT), mean_w2(SCHEME_DTR)
    assert abs(dtr / dt - 1.0) < 0.03, (dt, dtr)
