"""Pins for the oracle's model layer: the update rule of Eq. (1), the flat start,
lattice invariants, the h -> -h symmetry and the canonical exchange layout."""
import numpy as np
import pytest


def _evolved(oracle, L, seed, n_mcs, p=0.7, q=0.2):
    X, Y = oracle.flat(L)
    oracle.seq_rs(X, Y, p, q, seed, 0, n_mcs)
    return X, Y


def test_flat_start_every_site_is_extremal(oracle):
    L = 16
    X, Y = oracle.flat(L)
    assert oracle.invariants(X, Y) == 0
    for y in range(L):
        for x in range(L):
            # h = (x+y) mod 2: even sites sit below all four neighbours.
            assert oracle.site_kind(X, Y, x, y) == (1 if (x + y) % 2 == 0 else -1)


def test_flat_start_roughness_closed_form(oracle):
    for L in (4, 16, 64):
        X, Y = oracle.flat(L)
        s1, s2, hmax = oracle.w2_sums(X, Y)
        N = L * L
        assert (s1, s2, hmax) == (N // 2, N // 2, 1)
        assert oracle.w2(X, Y) == 0.25


def test_single_deposition_closed_form(oracle):
    L = 16
    N = L * L
    X, Y = oracle.flat(L)
    r, kind = oracle.attempt(X, Y, 2, 0, 1.0, 0.0, 0)
    assert (r, kind) == (1, 1)
    assert oracle.invariants(X, Y) == 0
    s1, s2, _ = oracle.w2_sums(X, Y)
    # heights relative to h(0,0)=0: one even site rose from 0 to 2.
    assert (s1, s2) == (N // 2 + 2, N // 2 + 4)
    expect = (N * (N // 2 + 4) - (N // 2 + 2) ** 2) / N**2
    assert oracle.w2(X, Y) == pytest.approx(expect, rel=0, abs=1e-15)
    # the deposited site is now a local maximum, its neighbours are not minima
    assert oracle.site_kind(X, Y, 2, 0) == -1


def test_attempt_respects_probabilities(oracle):
    X, Y = oracle.flat(8)
    X0, Y0 = X.copy(), Y.copy()
    # minimum at an even site, p = 0: never
    assert oracle.attempt(X, Y, 0, 0, 0.0, 1.0, 0) == (0, 1)
    # maximum at an odd site, q = 0: never
    assert oracle.attempt(X, Y, 1, 0, 1.0, 0.0, 0) == (0, -1)
    assert np.array_equal(X, X0) and np.array_equal(Y, Y0)
    # p = 0.5: u = 2^31 - 1 accepted, u = 2^31 rejected
    assert oracle.attempt(X, Y, 0, 0, 0.5, 0.0, 2**31)[0] == 0
    assert oracle.attempt(X, Y, 0, 0, 0.5, 0.0, 2**31 - 1)[0] == 1


def test_frozen_when_p_and_q_vanish(oracle):
    L = 64
    X, Y = _evolved(oracle, L, 5, 3)
    X0, Y0 = X.copy(), Y.copy()
    assert oracle.seq_rs(X, Y, 0.0, 0.0, 1, 0, 2) == 0
    prm = oracle.Params(L=L, p=0.0, q=0.0, seed=1, Bx=16, By=16)
    assert oracle.dtrdt_run(X, Y, prm, 0, 2)[0] == 0
    assert np.array_equal(X, X0) and np.array_equal(Y, Y0)


def test_kpz_first_sweep_only_deposits(oracle):
    L = 32
    X, Y = oracle.flat(L)
    net = oracle.seq_rs(X, Y, 1.0, 0.0, 3, 0, 1)
    s1, _, _ = oracle.w2_sums(X, Y)
    assert net > 0
    # absolute heights only grow when q = 0; with h(0,0) as reference the sum
    # still changes by 2 per deposition away from (0,0).
    assert oracle.invariants(X, Y) == 0


@pytest.mark.parametrize("which", ["seq", "dtrdt"])
def test_height_reflection_symmetry(oracle, which):
    """h -> -h maps minima to maxima: complementing every slope bit and swapping
    (p, q) must give exactly the complemented trajectory, because every attempt
    draws the same site and the same uniform."""
    L = 64
    p, q = 0.7, 0.2
    A_X, A_Y = _evolved(oracle, L, 11, 2)
    X1, Y1 = A_X.copy(), A_Y.copy()
    X2, Y2 = (1 - A_X).astype(np.uint8), (1 - A_Y).astype(np.uint8)
    if which == "seq":
        n1 = oracle.seq_rs(X1, Y1, p, q, 21, 5, 3)
        n2 = oracle.seq_rs(X2, Y2, q, p, 21, 5, 3)
    else:
        n1 = oracle.dtrdt_run(X1, Y1, oracle.Params(L=L, p=p, q=q, seed=21, Bx=32, By=16), 5, 3)[0]
        n2 = oracle.dtrdt_run(X2, Y2, oracle.Params(L=L, p=q, q=p, seed=21, Bx=32, By=16), 5, 3)[0]
    assert n1 == -n2 and n1 != 0
    assert np.array_equal(X2, 1 - X1) and np.array_equal(Y2, 1 - Y1)


def test_invariants_hold_after_dynamics(oracle):
    L = 64
    for p, q in ((1.0, 0.0), (0.95, 0.05), (0.5, 0.5)):
        X, Y = _evolved(oracle, L, 2, 4, p, q)
        assert oracle.invariants(X, Y) == 0
        for prm in (oracle.Params(L=L, p=p, q=q, seed=9, Bx=32, By=32),
                    oracle.Params(L=L, p=p, q=q, seed=9, Bx=32, By=16, cx=8, cy=8)):
            oracle.dtrdt_run(X, Y, prm, 0, 3)
            assert oracle.invariants(X, Y) == 0


def test_invariant_checker_detects_planted_mistakes(oracle):
    X, Y = _evolved(oracle, 32, 4, 2)
    assert oracle.invariants(X, Y) == 0
    Xb = X.copy()
    Xb[5, 7] ^= 1
    assert oracle.invariants(Xb, Y) == 1 | 4
    Yb = Y.copy()
    Yb[3, 9] ^= 1
    assert oracle.invariants(X, Yb) == 2 | 4
    # a "flip" that forgets the partner x-bit keeps columns balanced only in Y
    Xc, Yc = X.copy(), Y.copy()
    for y in range(32):
        for x in range(32):
            if oracle.site_kind(Xc, Yc, x, y) == 1:
                Xc[y, x] ^= 1
                Yc[y, x] ^= 1
                Yc[(y + 1) % 32, x] ^= 1
                break
        else:
            continue
        break
    assert oracle.invariants(Xc, Yc) & 1


def test_canonical_layout(oracle):
    # flat 4x4 block: sites with x+y odd carry X = Y = 1 at bit pairs
    # 2*(4*y+x): indices 1,3,4,6,9,11,12,14 -> 0x33CC33CC.
    X, Y = oracle.flat(8)
    w = oracle.pack_canonical(X, Y)
    assert w.shape == (4,)
    assert all(int(v) == 0x33CC33CC for v in w)
    Xr, Yr = _evolved(oracle, 32, 8, 3)
    w = oracle.pack_canonical(Xr, Yr)
    X2, Y2 = oracle.unpack_canonical(w, 32)
    assert np.array_equal(X2, Xr) and np.array_equal(Y2, Yr)
    # word (1,2) of a 32-lattice holds sites x in 4..7, y in 8..11
    i = 2 * (32 // 4) + 1
    v = int(w[i])
    for yy in range(4):
        for xx in range(4):
            b = 2 * (4 * yy + xx)
            assert (v >> b) & 1 == Xr[8 + yy, 4 + xx]
            assert (v >> (b + 1)) & 1 == Yr[8 + yy, 4 + xx]


def test_replica_seeds_distinct(oracle):
    seeds = {oracle.replica_seed(1, r) for r in range(4096)}
    assert len(seeds) == 4096
    assert oracle.replica_seed(1, 0) != oracle.replica_seed(2, 0)
