"""Pins of the oracle's two-time autocorrelations (Sec. 2: C(t,s) of Eq. (5),
its slope form C_s and height form C_h).

* t = s: C_h(s,s) = W^2(s) exactly (the identity the paper states after
  Eq. (6)), and C_s(s,s) = 1/4 on any valid slope field (each row and column
  holds L/2 up-slopes, so <n> = 1/2 and <n n> = 1/2).
* Brute force: heights integrated the other way round (along row 0, then up
  each column) with numpy, covariance in Python integers.
* Closed form: one deposition on the flat start gives C_h = C_s = 1/4 - 1/N.
* Symmetries: swapping t and s; h -> -h (complementing every bit) of one
  lattice flips the sign of both C's, of both lattices leaves them unchanged;
  a common translation of both lattices leaves them unchanged.
* Cauchy-Schwarz: C_h(t,s)^2 <= W^2(t) W^2(s).
"""
import numpy as np
import pytest

from oracle import Params


def _evolved(oracle, L, p, q, seed, mcs, Bx=None):
    X, Y = oracle.flat(L)
    B = Bx or min(64, L // 2)
    prm = Params(L=L, p=p, q=q, seed=seed, Bx=B, By=B)
    oracle.dtrdt_run(X, Y, prm, 0, mcs)
    return X, Y


def _brute(Xt, Yt, Xs, Ys):
    def heights(X, Y):
        L = X.shape[0]
        row0 = np.concatenate([[0], np.cumsum(2 * X[0, 1:].astype(np.int64) - 1)])
        cols = np.vstack([np.zeros((1, L), np.int64), np.cumsum(2 * Y[1:, :].astype(np.int64) - 1, axis=0)])
        return row0[None, :] + cols

    ht, hs = heights(Xt, Yt), heights(Xs, Ys)
    N = ht.size
    cross = int((ht * hs).sum())
    st, ss = int(ht.sum()), int(hs.sum())
    occ = int((Xt & Xs).sum()) + int((Yt & Ys).sum())
    mt = int(Xt.sum()) + int(Yt.sum())
    ms = int(Xs.sum()) + int(Ys.sum())
    return {"sum_ht": st, "sum_hs": ss, "cross": cross, "occ": occ, "m_t": mt, "m_s": ms,
            "num_h": N * cross - st * ss, "num_s": 2 * N * occ - mt * ms}


@pytest.fixture(scope="module")
def pair(oracle):
    L = 32
    Xs, Ys = _evolved(oracle, L, 0.95, 0.05, 7, 3, Bx=8)
    Xt, Yt = Xs.copy(), Ys.copy()
    oracle.dtrdt_run(Xt, Yt, Params(L=L, p=0.95, q=0.05, seed=7, Bx=8, By=8), 3, 5)
    return Xt, Yt, Xs, Ys


def test_equal_times_give_w2(oracle):
    for L, p, q, seed, mcs in [(16, 1.0, 0.0, 1, 3), (32, 0.95, 0.05, 2, 4), (64, 0.5, 0.5, 3, 6)]:
        X, Y = _evolved(oracle, L, p, q, seed, mcs, Bx=8)
        a = oracle.two_time(X, Y, X, Y)
        s1, s2, _ = oracle.w2_sums(X, Y)
        assert a["sum_ht"] == a["sum_hs"] == s1
        assert a["cross"] == s2
        assert a["c_h"] == oracle.w2(X, Y)
        assert a["c_s"] == 0.25


def test_against_column_first_brute_force(oracle, pair):
    Xt, Yt, Xs, Ys = pair
    a = oracle.two_time(Xt, Yt, Xs, Ys)
    b = _brute(Xt, Yt, Xs, Ys)
    assert a["sum_ht"] == b["sum_ht"] and a["sum_hs"] == b["sum_hs"]
    assert a["cross"] == b["cross"]
    assert a["occ_x"] + a["occ_y"] == b["occ"]
    assert a["m_t"] == b["m_t"] and a["m_s"] == b["m_s"]
    N = Xt.size
    assert a["c_h"] == pytest.approx(b["num_h"] / N**2, rel=1e-15, abs=1e-15)
    assert a["c_s"] == pytest.approx(b["num_s"] / (2 * N) ** 2, rel=1e-15, abs=1e-15)
    # the lattices really differ, so the cross term is not a disguised W^2
    assert a["cross"] != oracle.w2_sums(Xt, Yt)[1]


@pytest.mark.parametrize("site", [(0, 0), (6, 4), (31, 31)])
def test_one_deposition_closed_form(oracle, site):
    L = 32
    N = L * L
    Xs, Ys = oracle.flat(L)
    Xt, Yt = Xs.copy(), Ys.copy()
    x, y = site
    assert (x + y) % 2 == 0  # a minimum of the flat start
    Xt[y, x] ^= 1
    Xt[y, (x + 1) % L] ^= 1
    Yt[y, x] ^= 1
    Yt[(y + 1) % L, x] ^= 1
    assert oracle.invariants(Xt, Yt) == 0
    a = oracle.two_time(Xt, Yt, Xs, Ys)
    assert a["c_h"] == 0.25 - 1.0 / N
    assert a["c_s"] == 0.25 - 1.0 / N
    assert N * a["cross"] - a["sum_ht"] * a["sum_hs"] == N * N // 4 - N


def test_symmetries(oracle, pair):
    Xt, Yt, Xs, Ys = pair
    a = oracle.two_time(Xt, Yt, Xs, Ys)
    b = oracle.two_time(Xs, Ys, Xt, Yt)
    assert (b["cross"], b["sum_ht"], b["sum_hs"]) == (a["cross"], a["sum_hs"], a["sum_ht"])
    assert b["c_h"] == a["c_h"] and b["c_s"] == a["c_s"]
    # h -> -h of one lattice: both covariances change sign, exactly
    c = oracle.two_time(1 - Xt, 1 - Yt, Xs, Ys)
    assert c["c_h"] == -a["c_h"] and c["c_s"] == -a["c_s"]
    d = oracle.two_time(1 - Xt, 1 - Yt, 1 - Xs, 1 - Ys)
    assert d["c_h"] == a["c_h"] and d["c_s"] == a["c_s"]
    # common translation of both lattices (the reference site h(0,0) moves)
    sh = (5, 11)
    e = oracle.two_time(*(np.ascontiguousarray(np.roll(v, sh, axis=(0, 1))) for v in (Xt, Yt, Xs, Ys)))
    assert e["c_h"] == a["c_h"] and e["c_s"] == a["c_s"]


def test_cauchy_schwarz(oracle, pair):
    Xt, Yt, Xs, Ys = pair
    a = oracle.two_time(Xt, Yt, Xs, Ys)
    assert a["c_h"] ** 2 <= oracle.w2(Xt, Yt) * oracle.w2(Xs, Ys)
    assert a["c_h"] > 0  # two states 5 MCS apart are positively correlated


def test_planted_sign_error_is_caught(oracle, pair):
    """A plausible slip (dropping the h(0,y) cross term) changes the value:
    the brute-force comparison above would catch it."""
    Xt, Yt, Xs, Ys = pair
    b = _brute(Xt, Yt, Xs, Ys)
    # recompute the cross sum without the column offsets of the s lattice
    L = Xt.shape[0]
    rt = np.cumsum(np.concatenate([np.zeros((L, 1), np.int64), 2 * Xt[:, 1:].astype(np.int64) - 1], axis=1), axis=1)
    h0t = np.concatenate([[0], np.cumsum(2 * Yt[1:, 0].astype(np.int64) - 1)])
    rs = np.cumsum(np.concatenate([np.zeros((L, 1), np.int64), 2 * Xs[:, 1:].astype(np.int64) - 1], axis=1), axis=1)
    wrong = int(((h0t[:, None] + rt) * rs).sum())
    assert wrong != b["cross"]
