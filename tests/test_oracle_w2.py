"""Pins for the exact roughness W^2 of Eq. (3) (mean taken over the L^2 sites).

The sums are checked against closed forms (in test_oracle_model.py), against a
second integration path (column first), against translation and reflection
invariance, and against a direct numpy evaluation of the definition for a
field built from known heights."""
import numpy as np
import pytest


def test_integration_order_independent(oracle):
    for L, p, q, n in ((32, 1.0, 0.0, 5), (64, 0.7, 0.2, 3), (128, 0.5, 0.5, 2)):
        X, Y = oracle.flat(L)
        oracle.seq_rs(X, Y, p, q, 17, 0, n)
        s1a, s2a, _ = oracle.w2_sums(X, Y)
        s1b, s2b = oracle.w2_sums_colfirst(X, Y)
        assert (s1a, s2a) == (s1b, s2b)


def test_translation_and_reflection_invariance(oracle):
    L = 64
    X, Y = oracle.flat(L)
    oracle.seq_rs(X, Y, 0.95, 0.05, 4, 0, 6)
    w = oracle.w2(X, Y)
    assert w > 0.3
    for dx, dy in ((1, 0), (0, 1), (5, 9), (63, 17)):
        Xs = np.ascontiguousarray(np.roll(X, (dy, dx), axis=(0, 1)))
        Ys = np.ascontiguousarray(np.roll(Y, (dy, dx), axis=(0, 1)))
        assert oracle.w2(Xs, Ys) == pytest.approx(w, rel=1e-14)
    Xc = (1 - X).astype(np.uint8)
    Yc = (1 - Y).astype(np.uint8)
    assert oracle.w2(Xc, Yc) == pytest.approx(w, rel=1e-14)


def test_matches_definition_on_known_heights(oracle):
    """Build a lattice from an explicit height field and evaluate Eq. (3)
    directly in exact integer arithmetic."""
    L = 32
    X, Y = oracle.flat(L)
    oracle.seq_rs(X, Y, 0.8, 0.2, 5, 0, 4)
    # heights by explicit summation of slopes, independent loops
    h = np.zeros((L, L), dtype=np.int64)
    for y in range(1, L):
        h[y, 0] = h[y - 1, 0] + (2 * int(Y[y, 0]) - 1)
    for y in range(L):
        for x in range(1, L):
            h[y, x] = h[y, x - 1] + (2 * int(X[y, x]) - 1)
    s1 = int(h.sum())
    s2 = int((h * h).sum())
    N = L * L
    assert oracle.w2_sums(X, Y)[:2] == (s1, s2)
    exact = (N * s2 - s1 * s1) / N**2
    direct = float(np.mean(h.astype(float) ** 2) - np.mean(h.astype(float)) ** 2)
    assert oracle.w2(X, Y) == pytest.approx(exact, rel=1e-15)
    assert oracle.w2(X, Y) == pytest.approx(direct, rel=1e-12)


def test_large_sums_need_128_bits(oracle):
    """S2 in 128 bits: the combination N*S2 - S1^2 exceeds 64 bits for the
    paper's sizes; the helper must not truncate."""
    L = 2**17
    N = L * L
    s1 = 3 * N
    s2 = 10 * N  # mean 3, mean square 10 -> W^2 = 1
    assert oracle.w2_from_sums(L, s1, s2) == 1.0
    s2 = 2**70 + 12345
    w = oracle.w2_from_sums(L, 0, s2)
    assert w == pytest.approx(s2 / N, rel=1e-15)
