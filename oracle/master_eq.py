"""Exact master equations of the octahedron model on the 4x4 torus (test infrastructure).

Only the test-suite imports this module.  It is an independent statement of
the dynamics, used to pin the C oracle:

* It is written in terms of heights, not slope bits.  A site is a local
  minimum when all four neighbours stand one unit higher.  A deposition
  (probability p) raises it by two.  Removals at local maxima (probability q)
  mirror this.  This is the octahedron model of Sec. 2.1; the slope-bit
  rule of Eq. (1) is its lattice-gas image, and the C oracle implements that
  image.  Agreement of the two pins the slope-bit reading.
* States are slope configurations (heights modulo a global shift), encoded
  from the heights, and enumerated by breadth-first search from the flat
  start h = (x+y) mod 2.
* ``rs_attempt_matrix``: one random-sequential attempt (uniform site).  One
  MCS is L^2 = 16 attempts (the paper's MCS definition).
* ``dtrdt_mcs_matrix``: one MCS of DTrDT with sub-tiles 2x2 and thread cells
  2x2 sites.  Each sub-cell is then a single site, so the only randomness is
  the origin (uniform on the 16 sites), the order of the four sets (uniform
  over the 24 permutations), the block-level domain set of each of the four
  collective steps (uniform, drawn with replacement) and the acceptance.

Acceptance probabilities are the rounded P32/2^32 of the oracle's threshold
reading; the rounding changes p by less than 2^-32.
"""
from __future__ import annotations

import itertools
from collections import deque

import numpy as np

L = 4


def heights_flat() -> np.ndarray:
    y, x = np.mgrid[0:L, 0:L]
    return ((x + y) % 2).astype(np.int64)


def encode(h: np.ndarray) -> int:
    """Slope code of a height field: bit (y*L+x) = [h(x,y)-h(x-1,y) = +1],
    bit 16+(y*L+x) = [h(x,y)-h(x,y-1) = +1]."""
    dx = h - np.roll(h, 1, axis=1)
    dy = h - np.roll(h, 1, axis=0)
    assert np.all(np.abs(dx) == 1) and np.all(np.abs(dy) == 1)
    code = 0
    for y in range(L):
        for x in range(L):
            if dx[y, x] == 1:
                code |= 1 << (y * L + x)
            if dy[y, x] == 1:
                code |= 1 << (16 + y * L + x)
    return code


def decode(code: int) -> np.ndarray:
    """Heights with h(0,0) = 0 from a slope code."""
    h = np.zeros((L, L), dtype=np.int64)
    for y in range(L):
        if y > 0:
            h[y, 0] = h[y - 1, 0] + (1 if (code >> (16 + y * L)) & 1 else -1)
        for x in range(1, L):
            h[y, x] = h[y, x - 1] + (1 if (code >> (y * L + x)) & 1 else -1)
    return h


def code_to_bits(code: int):
    """Slope code -> (X, Y) uint8 arrays [y, x] in the oracle's convention."""
    X = np.zeros((L, L), dtype=np.uint8)
    Y = np.zeros((L, L), dtype=np.uint8)
    for y in range(L):
        for x in range(L):
            X[y, x] = (code >> (y * L + x)) & 1
            Y[y, x] = (code >> (16 + y * L + x)) & 1
    return X, Y


def bits_to_code(X: np.ndarray, Y: np.ndarray) -> int:
    code = 0
    for y in range(L):
        for x in range(L):
            code |= int(X[y, x]) << (y * L + x)
            code |= int(Y[y, x]) << (16 + y * L + x)
    return code


def _neighbours(h: np.ndarray, x: int, y: int):
    return (h[y, (x + 1) % L], h[y, (x - 1) % L], h[(y + 1) % L, x], h[(y - 1) % L, x])


def kind(h: np.ndarray, x: int, y: int) -> int:
    """+1 local minimum (all neighbours one higher), -1 local maximum, 0 otherwise."""
    nb = _neighbours(h, x, y)
    if all(v == h[y, x] + 1 for v in nb):
        return +1
    if all(v == h[y, x] - 1 for v in nb):
        return -1
    return 0


def flipped(code: int, x: int, y: int) -> int | None:
    h = decode(code)
    k = kind(h, x, y)
    if k == 0:
        return None
    h = h.copy()
    h[y, x] += 2 * k
    return encode(h)


def reachable_states():
    """All slope configurations reachable from the flat start by single-site
    depositions/removals (BFS).  Returns (codes list, index dict)."""
    start = encode(heights_flat())
    seen = {start: 0}
    order = [start]
    dq = deque([start])
    while dq:
        c = dq.popleft()
        for y in range(L):
            for x in range(L):
                n = flipped(c, x, y)
                if n is not None and n not in seen:
                    seen[n] = len(order)
                    order.append(n)
                    dq.append(n)
    return order, seen


def site_matrix(states, index, x: int, y: int, pe: float, qe: float) -> np.ndarray:
    """Transition matrix of one attempt at a fixed site (row-stochastic)."""
    n = len(states)
    A = np.zeros((n, n))
    for i, c in enumerate(states):
        h = decode(c)
        k = kind(h, x, y)
        if k == 0:
            A[i, i] = 1.0
            continue
        prob = pe if k > 0 else qe
        j = index[flipped(c, x, y)]
        A[i, j] += prob
        A[i, i] += 1.0 - prob
    return A


def site_matrices(states, index, pe: float, qe: float):
    return {(x, y): site_matrix(states, index, x, y, pe, qe) for y in range(L) for x in range(L)}


def rs_attempt_matrix(states, index, pe: float, qe: float) -> np.ndarray:
    A = site_matrices(states, index, pe, qe)
    return sum(A.values()) / (L * L)


def dtrdt_mcs_matrix(states, index, pe: float, qe: float) -> np.ndarray:
    """One DTrDT MCS with Bx = By = 2, cx = cy = 2 on the 4x4 torus."""
    A = site_matrices(states, index, pe, qe)
    n = len(states)
    # M[(x0, y0)]: one device step on the 2x2 sub-tile at (x0, y0): four
    # collective steps, each attempting the site of a uniformly drawn set d.
    M = {}
    for y0 in range(L):
        for x0 in range(L):
            avg = sum(A[((x0 + dx) % L, (y0 + dy) % L)] for dy in (0, 1) for dx in (0, 1)) / 4.0
            M[(x0, y0)] = np.linalg.matrix_power(avg, 4)
    T = np.zeros((n, n))
    for oy in range(L):
        for ox in range(L):
            D = [M[((ox + 2 * (s & 1)) % L, (oy + 2 * (s >> 1)) % L)] for s in range(4)]
            T += _sum_over_orders(D) / 24.0
    return T / (L * L)


def _sum_over_orders(D):
    """Sum over all 24 orders (s0,s1,s2,s3) of the products D[s0] D[s1] D[s2] D[s3].

    Computed by recursion on the set of factors already applied: the sum over
    orders of a set S equals the sum over its last element a of
    (sum over orders of S minus a) times D[a]."""
    f = {}
    for size in range(1, 5):
        for S in itertools.combinations(range(4), size):
            if size == 1:
                f[S] = D[S[0]]
                continue
            acc = 0
            for a in S:
                rest = tuple(b for b in S if b != a)
                acc = acc + f[rest] @ D[a]
            f[S] = acc
    return f[(0, 1, 2, 3)]


def dtrdt_mcs_matrix_by_orders(states, index, pe: float, qe: float) -> np.ndarray:
    """The same matrix with an explicit loop over the 24 permutations (slow; for
    checking the recursion)."""
    A = site_matrices(states, index, pe, qe)
    n = len(states)
    T = np.zeros((n, n))
    for oy in range(L):
        for ox in range(L):
            Ms = {}
            for s in range(4):
                x0, y0 = (ox + 2 * (s & 1)) % L, (oy + 2 * (s >> 1)) % L
                avg = sum(A[((x0 + dx) % L, (y0 + dy) % L)] for dy in (0, 1) for dx in (0, 1)) / 4
                Ms[s] = np.linalg.matrix_power(avg, 4)
            for perm in itertools.permutations(range(4)):
                P = np.eye(n)
                for s in perm:
                    P = P @ Ms[s]
                T += P / 24.0
    return T / (L * L)


def distribution(T: np.ndarray, steps: int, n_states: int) -> np.ndarray:
    """pi_0 T^steps from the flat start (state 0)."""
    pi = np.zeros(n_states)
    pi[0] = 1.0
    return pi @ np.linalg.matrix_power(T, steps)


def g_test(counts: np.ndarray, probs: np.ndarray, min_expected: float = 5.0):
    """Likelihood-ratio (G) goodness-of-fit test; small expected bins are pooled.
    Returns (G, dof, p_value)."""
    from scipy.stats import chi2
    total = counts.sum()
    exp = probs * total
    big = exp >= min_expected
    obs_b = list(counts[big])
    exp_b = list(exp[big])
    if (~big).any():
        obs_b.append(counts[~big].sum())
        exp_b.append(exp[~big].sum())
    obs_b = np.asarray(obs_b, dtype=float)
    exp_b = np.asarray(exp_b, dtype=float)
    if counts[exp == 0].sum() > 0:
        # a configuration the master equation forbids was observed
        return float("inf"), len(obs_b) - 1, 0.0
    nz = obs_b > 0
    G = 2.0 * np.sum(obs_b[nz] * np.log(obs_b[nz] / exp_b[nz]))
    dof = len(obs_b) - 1
    return G, dof, float(chi2.sf(G, dof))
