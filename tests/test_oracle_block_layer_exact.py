"""Exact pins of the oracle's block layer with several thread cells per sub-tile.

The 4x4 master equations (test_oracle_master_eq.py) run at thread cells of
2x2 sites with one cell per sub-tile, where no site bits are drawn and where
the order of the DTrDB phases cannot matter.  The tests here close those gaps:

* the site of every thread cell's attempt equals an independent Python
  statement of the stated random-number reading (the site field of the
  SITE / SITE_DB word of the cell's group, the block's set draw and, for
  DTrDTr, its block origin), at the cell shapes the GPU runs;
* the offsets of neighbouring cells (same band, next band column, next TC
  row, next group, next collective step) are jointly uniform and
  independent (G-test on the joint table);
* the distribution of the lattice after one collective step of a sub-tile
  with several cells equals the exact distribution, enumerated here over the
  block draws, the cells' sites and the acceptances, for DT (Sec. 3.1,
  single-hit block layer), DTrDB with delayed borders (Sec. 3.1: bulk, then
  borders, then corners) and DTrDTr (Sec. 4.1.2: the cell grid moved to a
  random origin before every collective update);
* two planted mistakes fail: cells that share site bits, and corner attempts
  carried out before border attempts."""
import itertools
import math

import numpy as np
import pytest

from oracle import master_eq as me

TAG_SET, TAG_SITE, TAG_SITE_DB, TAG_BORG = 2, 3, 8, 9
P_MIN = 1e-4


# ------------------------------------------------- independent statement ---

def _log2(v):
    k = int(round(math.log2(v)))
    assert 1 << k == v
    return k


def _key(seed):
    return [seed & 0xFFFFFFFF, seed >> 32]


def stated_sites(oracle, prm, t, k, T, s):
    """Local sites of every thread cell's attempt in collective step s, from
    the stated reading: a band is one TC row, BW = min(32, Bx) sites wide;
    a group is four TC rows of one band column, g = (c//4)*(Bx/BW) + band
    column, m = c % 4; the cell's offset sits in word m of its group's site
    word at bit fw*j + (s % spw)*(fw/spw), low bits x then y."""
    Bx, By, cx, cy = prm.Bx, prm.By, prm.cx, prm.cy
    db = prm.scheme in (oracle.SCHEME_DB, oracle.SCHEME_DB_IGNORE)
    dtr = prm.scheme == oracle.SCHEME_DTR
    BW = min(32, Bx)
    tpb = BW // cx
    band_cols = Bx // BW
    ux, uy = (cx, cy) if db else (cx // 2, cy // 2)
    bx, by = _log2(ux), _log2(uy)
    bpt = bx + by
    fw = 32 // tpb
    spw = 2 if (bpt > 0 and 2 * bpt <= fw) else 1
    key = _key(prm.seed)
    tag = TAG_SITE_DB if db else TAG_SITE
    dx = dy = 0
    c0 = r0 = 0
    if not db:
        sw = oracle.philox([t, k | ((s // 64) << 2), T, TAG_SET << 28], key)
        d = (int(sw[(s % 64) // 16]) >> (2 * (s % 16))) & 3
        dx, dy = d & 1, d >> 1
        c0, r0 = dx * ux, dy * uy
        if dtr:
            bw = oracle.philox([t, k | ((s // 16) << 2), T, TAG_BORG << 28], key)
            byte = (int(bw[(s % 16) // 4]) >> (8 * (s % 4))) & 0xFF
            ax, ay = byte & (cx - 1), (byte >> 4) & (cy - 1)
            c0, r0 = (ax + c0) % cx, (ay + r0) % cy
    n_a, n_c = Bx // cx, By // cy
    lx = np.zeros(n_a * n_c, dtype=np.int64)
    ly = np.zeros(n_a * n_c, dtype=np.int64)
    words = {}
    for c in range(n_c):
        for a in range(n_a):
            g = (c // 4) * band_cols + a // tpb
            j, m = a % tpb, c % 4
            rx = ry = 0
            if bpt > 0:
                if g not in words:
                    words[g] = oracle.philox([t, k | ((s // spw) << 2), T, (tag << 28) | g], key)
                r = (int(words[g][m]) >> (fw * j + (s % spw) * (fw // spw))) & ((1 << bpt) - 1)
                rx, ry = r & (ux - 1), r >> bx
            lx[c * n_a + a] = (a * cx + c0 + rx) % Bx
            ly[c * n_a + a] = (c * cy + r0 + ry) % By
    return lx, ly


SHAPES = [  # (Bx, By, cx, cy, scheme)
    (64, 32, 4, 4, 0), (64, 64, 8, 8, 0), (64, 64, 16, 8, 0), (64, 64, 16, 16, 0), (32, 64, 8, 16, 0),
    (64, 32, 8, 4, 0), (32, 32, 4, 8, 0), (64, 32, 4, 4, 1), (64, 64, 8, 8, 1), (64, 64, 16, 16, 1),
    (64, 32, 4, 4, 3), (64, 64, 8, 8, 3), (128, 16, 32, 16, 0),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda v: "B{}x{}_TC{}x{}_s{}".format(*v))
def test_sites_follow_the_stated_fields(oracle, shape):
    Bx, By, cx, cy, scheme = shape
    prm = oracle.Params(L=4 * max(Bx, By), p=0.5, q=0.5, seed=(7 << 32) + 5, Bx=Bx, By=By, cx=cx, cy=cy,
                        scheme=scheme)
    assert oracle.check_params(prm)
    for (t, k, T, s) in ((0, 0, 0, 0), (3, 2, 5, 1), (11, 3, 2, cx * cy - 1), (5, 1, 7, 6)):
        if s >= cx * cy:
            continue
        lx, ly = oracle.subtile_step_sites(prm, t, k, T, s)
        ex, ey = stated_sites(oracle, prm, t, k, T, s)
        assert np.array_equal(lx, ex) and np.array_equal(ly, ey), (t, k, T, s)


def test_planted_shared_site_bits_break_the_statement(oracle):
    prm = oracle.Params(L=128, p=0.5, q=0.5, seed=5, Bx=64, By=32)
    with oracle.planted(1):
        lx, ly = oracle.subtile_step_sites(prm, 3, 2, 5, 1)
    ex, ey = stated_sites(oracle, prm, 3, 2, 5, 1)
    assert not (np.array_equal(lx, ex) and np.array_equal(ly, ey))


# ------------------------------------------ joint offsets of neighbours ---

def _joint_g_test(a, b, n_values):
    table = np.zeros((n_values, n_values))
    np.add.at(table, (a, b), 1)
    return me.g_test(table.reshape(-1), np.full(n_values * n_values, 1.0 / n_values ** 2))


def _offsets(oracle, prm, n_calls):
    """Offsets (index inside the sub-cell) of every thread cell over n_calls
    collective steps drawn over MCS, device steps, tiles and step indices."""
    ux, uy = prm.cx // 2, prm.cy // 2
    n_a, n_c = prm.Bx // prm.cx, prm.By // prm.cy
    out = []
    steps = prm.cx * prm.cy
    for i in range(n_calls):
        block, s = i // steps, i % steps  # consecutive calls: steps s, s+1 of one sub-tile
        t, k, T = block // 20, (block // 5) % 4, 3 + block % 5
        lx, ly = oracle.subtile_step_sites(prm, t, k, T, s)
        out.append(((ly % uy) * ux + lx % ux).reshape(n_c, n_a))
    return np.array(out)  # [call, TC row, TC column]


CELLS = [(4, 4, 1600), (8, 8, 1200), (16, 8, 2800)]


@pytest.mark.parametrize("cx,cy,n_calls", CELLS, ids=lambda v: str(v))
def test_neighbouring_cells_draw_independent_offsets(oracle, cx, cy, n_calls):
    """Pairs of neighbouring cells: same band (j, j+1), across band columns
    (the last cell of one group and the first of the next), same band column
    in TC rows m, m+1 of a group and across group rows, and the same cell in
    collective steps s, s+1 (which share a site word when two steps are
    served by one field).  Each joint table must be uniform on A x A."""
    Bx, By = 64, 8 * cy
    prm = oracle.Params(L=2 * max(Bx, By), p=0.5, q=0.5, seed=99, Bx=Bx, By=By, cx=cx, cy=cy)
    A = (cx // 2) * (cy // 2)
    off = _offsets(oracle, prm, n_calls)
    tpb = 32 // cx
    pairs = {
        "band": (off[:, :, 0], off[:, :, 1]),
        "band_columns": (off[:, :, tpb - 1], off[:, :, tpb]),
        "rows": (off[:, 0, :], off[:, 1, :]),
        "groups": (off[:, 3, :], off[:, 4, :]),
        "steps": (off[:-1:2], off[1::2]),
    }
    for name, (a, b) in pairs.items():
        G, dof, pval = _joint_g_test(a.reshape(-1), b.reshape(-1), A)
        assert pval > P_MIN, (name, G, dof, pval)
    # Cells 0 and 1 of a band agree with probability 1/A; the planted mistake
    # (cells 2i, 2i+1 share bits) makes them always agree.
    same = np.mean(off[:, :, 0] == off[:, :, 1])
    n = off[:, :, 0].size
    assert abs(same - 1.0 / A) < 5 * np.sqrt((1.0 / A) * (1 - 1.0 / A) / n), same
    with oracle.planted(1):
        bad = _offsets(oracle, prm, 200)
    assert np.all(bad[:, :, 0] == bad[:, :, 1])


# ------------------------------------------- exact one-step distributions ---

def _kind(X, Y, x, y):
    """Eq. (1) on slope bits: +1 local minimum, -1 local maximum, 0 neither."""
    L = X.shape[0]
    xs, xn = X[y, x], X[y, (x + 1) % L]
    ys, yn = Y[y, x], Y[(y + 1) % L, x]
    if (xs, xn, ys, yn) == (0, 1, 0, 1):
        return 1
    if (xs, xn, ys, yn) == (1, 0, 1, 0):
        return -1
    return 0


def _flip(X, Y, x, y):
    L = X.shape[0]
    X[y, x] ^= 1
    X[y, (x + 1) % L] ^= 1
    Y[y, x] ^= 1
    Y[(y + 1) % L, x] ^= 1


def _state_key(X, Y):
    return np.packbits(np.concatenate([X.reshape(-1), Y.reshape(-1)])).tobytes()


def _add(dist, key, pr):
    dist[key] = dist.get(key, 0.0) + pr


def exact_dt_like(X0, Y0, x0, y0, Bx, By, cx, cy, pe, qe, origins):
    """Exact distribution after one collective step in which every cell
    attempts one uniform site of its active sub-cell, all decided on the
    state before the step.  origins: list of (weight, c0, r0) of the active
    sub-cell's first column / row in every cell (the block's draws)."""
    L = X0.shape[0]
    ux, uy = cx // 2, cy // 2
    dist = {}
    for w, c0, r0 in origins:
        per_cell = []
        for c in range(By // cy):
            for a in range(Bx // cx):
                outs = {}
                for ry in range(uy):
                    for rx in range(ux):
                        x = (x0 + (a * cx + c0 + rx) % Bx) % L
                        y = (y0 + (c * cy + r0 + ry) % By) % L
                        kd = _kind(X0, Y0, x, y)
                        pa = pe if kd > 0 else qe if kd < 0 else 0.0
                        if pa > 0:
                            outs[(x, y)] = outs.get((x, y), 0.0) + pa / (ux * uy)
                        outs[None] = outs.get(None, 0.0) + (1 - pa) / (ux * uy)
                per_cell.append(list(outs.items()))
        for combo in itertools.product(*per_cell):
            pr = w
            X, Y = X0.copy(), Y0.copy()
            for site, pc in combo:
                pr *= pc
                if site is not None:
                    _flip(X, Y, *site)
            if pr > 0:
                _add(dist, _state_key(X, Y), pr)
    return dist


def exact_db(X0, Y0, x0, y0, Bx, By, cx, cy, pe, qe, order=(0, 1, 2)):
    """Exact distribution after one DTrDB collective step with delayed
    borders: every cell attempts one uniform site of its whole cell; bulk
    attempts (x < cx-1 and y < cy-1) first, then border attempts (last column
    or last row), then the corner (cx-1, cy-1), each phase decided on the
    state the earlier ones left."""
    L = X0.shape[0]
    cells = [(a, c) for c in range(By // cy) for a in range(Bx // cx)]
    dist = {}
    w = 1.0 / (cx * cy) ** len(cells)
    for choice in itertools.product(range(cx * cy), repeat=len(cells)):
        att = []
        for (a, c), r in zip(cells, choice):
            rx, ry = r % cx, r // cx
            phase = (rx == cx - 1) + (ry == cy - 1)
            att.append((order.index(phase), (x0 + a * cx + rx) % L, (y0 + c * cy + ry) % L))
        att.sort()

        def branch(i, X, Y, pr):
            if i == len(att):
                _add(dist, _state_key(X, Y), pr)
                return
            _, x, y = att[i]
            kd = _kind(X, Y, x, y)
            pa = pe if kd > 0 else qe if kd < 0 else 0.0
            if pa > 0:
                X2, Y2 = X.copy(), Y.copy()
                _flip(X2, Y2, x, y)
                branch(i + 1, X2, Y2, pr * pa)
            if pa < 1:
                branch(i + 1, X, Y, pr * (1 - pa))

        branch(0, X0.copy(), Y0.copy(), w)
    return dist


def _sampled(oracle, prm, x0, y0, X0, Y0, n, seed0, chunk=20000):
    counts = {}
    for c in range(0, n, chunk):
        m = min(chunk, n - c)
        X, Y, _ = oracle.subtile_steps_many(prm, seed0 + c, m, 3, 1, 6, x0, y0, 1, X0, Y0)
        keys = np.packbits(np.concatenate([X.reshape(m, -1), Y.reshape(m, -1)], axis=1), axis=1)
        u, k = np.unique(keys, axis=0, return_counts=True)
        for row, cnt in zip(u, k):
            counts[row.tobytes()] = counts.get(row.tobytes(), 0) + int(cnt)
    return counts


def _compare(dist, counts):
    keys = list(dist) + [k for k in counts if k not in dist]
    probs = np.array([dist.get(k, 0.0) for k in keys])
    obs = np.array([counts.get(k, 0) for k in keys], dtype=float)
    assert abs(probs.sum() - 1.0) < 1e-9
    return me.g_test(obs, probs)


def _start_states(oracle, L):
    """The flat start (every site extremal) and a rough state after a few
    sweeps of sequential RS (O1)."""
    Xf, Yf = oracle.flat(L)
    Xr, Yr = oracle.flat(L)
    oracle.seq_rs(Xr, Yr, 0.6, 0.4, 4242, 0, 3)
    return [(Xf, Yf), (Xr, Yr)]


def _rates(oracle, p, q):
    return oracle.threshold32(p) / 2**32, oracle.threshold32(q) / 2**32


@pytest.mark.parametrize("Bx,By,x0,y0", [(8, 8, 3, 5), (4, 20, 6, 1)], ids=["4cells", "2groups"])
def test_dt_step_exact_distribution(oracle, Bx, By, x0, y0):
    """One DTrDT collective step (4x4-site cells, 2x2 sub-cells) on a sub-tile
    of four cells, and on a column of five cells spanning two groups."""
    L = 16 if By == 8 else 40
    p, q = 0.7, 0.45
    pe, qe = _rates(oracle, p, q)
    prm = oracle.Params(L=L, p=p, q=q, seed=1, Bx=Bx, By=By, cx=4, cy=4)
    origins = [(0.25, (d & 1) * 2, (d >> 1) * 2) for d in range(4)]
    for i, (X0, Y0) in enumerate(_start_states(oracle, L)):
        dist = exact_dt_like(X0, Y0, x0, y0, Bx, By, 4, 4, pe, qe, origins)
        counts = _sampled(oracle, prm, x0, y0, X0, Y0, 60000, 1000 + 100000 * i)
        G, dof, pval = _compare(dist, counts)
        assert pval > P_MIN, (i, G, dof, pval)
    # planted: cells 2i, 2i+1 share site bits (the four-cell sub-tile has two cells per band)
    if Bx == 8:
        X0, Y0 = _start_states(oracle, L)[0]
        with oracle.planted(1):
            counts = _sampled(oracle, prm, x0, y0, X0, Y0, 60000, 7)
        assert _compare(exact_dt_like(X0, Y0, x0, y0, Bx, By, 4, 4, pe, qe, origins), counts)[2] < 1e-12


def test_dtr_step_exact_distribution(oracle):
    """One DTrDTr collective step (4x4-site cells): the block draws the set and
    an origin (ax, ay) uniform in [0,4)^2; the cell grid wraps around the 8x8
    sub-tile."""
    L, Bx, By, x0, y0 = 16, 8, 8, 5, 2
    p, q = 0.6, 0.55
    pe, qe = _rates(oracle, p, q)
    prm = oracle.Params(L=L, p=p, q=q, seed=1, Bx=Bx, By=By, scheme=oracle.SCHEME_DTR)
    origins = [(1.0 / 64, (ax + 2 * (d & 1)) % 4, (ay + 2 * (d >> 1)) % 4)
               for d in range(4) for ax in range(4) for ay in range(4)]
    for i, (X0, Y0) in enumerate(_start_states(oracle, L)):
        dist = exact_dt_like(X0, Y0, x0, y0, Bx, By, 4, 4, pe, qe, origins)
        counts = _sampled(oracle, prm, x0, y0, X0, Y0, 60000, 5000 + 100000 * i)
        G, dof, pval = _compare(dist, counts)
        assert pval > P_MIN, (i, G, dof, pval)


DB_CASES = [(16, 4, 4, 2, 2, 1, 3), (16, 8, 4, 4, 4, 3, 5), (16, 4, 8, 4, 4, 6, 2)]


@pytest.mark.parametrize("L,Bx,By,cx,cy,x0,y0", DB_CASES, ids=["2x2cells_4", "4x4cells_side", "4x4cells_stacked"])
def test_db_step_exact_distribution(oracle, L, Bx, By, cx, cy, x0, y0):
    """One DTrDB collective step with both rates positive (delayed borders) on
    a sub-tile of several cells: four 2x2-site cells, and two 4x4-site cells
    side by side and stacked, where a corner attempt of one cell and a border
    attempt of its neighbour share a slope bit.  With 2x2 cells that happens
    in 1/16 of the steps, so there the planted corner-before-border order is
    rejected."""
    p, q = 0.65, 0.5
    pe, qe = _rates(oracle, p, q)
    prm = oracle.Params(L=L, p=p, q=q, seed=1, Bx=Bx, By=By, cx=cx, cy=cy, scheme=oracle.SCHEME_DB)
    states = _start_states(oracle, L)
    for i, (X0, Y0) in enumerate(states):
        dist = exact_db(X0, Y0, x0, y0, Bx, By, cx, cy, pe, qe)
        counts = _sampled(oracle, prm, x0, y0, X0, Y0, 60000, 9000 + 100000 * i)
        G, dof, pval = _compare(dist, counts)
        assert pval > P_MIN, (i, G, dof, pval)
    if cx != 2:
        return  # with 4x4 cells a corner meets a neighbour's border attempt in 1/256 of the steps
    # planted: corners before borders; fails against the exact delayed-border law
    X0, Y0 = states[0]
    exact = exact_db(X0, Y0, x0, y0, Bx, By, cx, cy, pe, qe)
    with oracle.planted(2):
        counts = _sampled(oracle, prm, x0, y0, X0, Y0, 60000, 11)
    assert _compare(exact, counts)[2] < 1e-12
    # and the two orders really are different laws on this start state
    swapped = exact_db(X0, Y0, x0, y0, Bx, By, cx, cy, pe, qe, order=(0, 2, 1))
    tv = 0.5 * sum(abs(exact.get(k, 0) - swapped.get(k, 0)) for k in set(exact) | set(swapped))
    assert tv > 0.02, tv


# ------------------------------------------------------------ tail streams ---

TAG_ACC = 4


def stated_ties(oracle, prm, t, k, T, s, x0, y0):
    """Tied candidates of collective step s of a sub-tile at the flat start,
    from the stated reading: every attempted site is extremal (a minimum iff
    x + y is even); the four leading bits of a cell's uniform are bit 4j+m of
    the four level words of its group (most significant first); the candidate
    ties iff they equal the four leading bits of P32 of its rate.  Each group
    takes words 0, 1, 2, ... of its own tail stream in order of position.
    Returns rows (stream group, word index, candidate group, position)."""
    lx, ly = stated_sites(oracle, prm, t, k, T, s)
    n_a = prm.Bx // prm.cx
    tpb = min(32, prm.Bx) // prm.cx
    band_cols = prm.Bx // min(32, prm.Bx)
    thr = {1: oracle.threshold32(prm.p) >> 28, -1: oracle.threshold32(prm.q) >> 28}
    key = _key(prm.seed)
    words = {}
    ties = []
    for i, (x, y) in enumerate(zip(lx, ly)):
        c, a = divmod(i, n_a)
        g = (c // 4) * band_cols + a // tpb
        pos = 4 * (a % tpb) + c % 4
        kind = 1 if (x0 + x + y0 + y) % 2 == 0 else -1
        if g not in words:
            words[g] = oracle.philox([t, k | ((s * 8) << 2), T, (TAG_ACC << 28) | g], key)
        hi = sum(((int(words[g][l]) >> pos) & 1) << (3 - l) for l in range(4))
        if hi == thr[kind]:
            ties.append((g, pos))
    ties.sort()
    rows, used = [], {}
    for g, pos in ties:
        rows.append((g, used.get(g, 0), g, pos))
        used[g] = used.get(g, 0) + 1
    return rows


def test_ties_take_their_groups_tail_words_in_position_order(oracle):
    """Four groups (64 cells of 4x4 sites in a 64 x 32 sub-tile), both rates
    random, step 0 from the flat start over 300 seeds: the oracle's record of
    the tail words its tied candidates take equals the stated reading; the
    planted mistake (all groups on group 0's stream) does not."""
    L, x0, y0 = 128, 5, 9
    n_ties = 0
    for seed in range(300):
        prm = oracle.Params(L=L, p=0.95, q=0.05, seed=seed, Bx=64, By=32)
        X0, Y0 = oracle.flat(L)
        with oracle.tie_log() as log:
            oracle.subtile_steps_many(prm, seed, 1, 3, 1, 6, x0, y0, 1, X0, Y0)
        want = stated_ties(oracle, prm, 3, 1, 6, 0, x0, y0)
        assert [tuple(r) for r in log.rows().tolist()] == want, seed
        n_ties += len(want)
    assert n_ties > 600
    prm = oracle.Params(L=L, p=0.95, q=0.05, seed=1, Bx=64, By=32)
    bad = 0
    for seed in range(40):
        prm = oracle.Params(L=L, p=0.95, q=0.05, seed=seed, Bx=64, By=32)
        X0, Y0 = oracle.flat(L)
        with oracle.planted(3), oracle.tie_log() as log:
            oracle.subtile_steps_many(prm, seed, 1, 3, 1, 6, x0, y0, 1, X0, Y0)
        bad += [tuple(r) for r in log.rows().tolist()] != stated_ties(oracle, prm, 3, 1, 6, 0, x0, y0)
    assert bad > 20


def test_tail_streams_are_uniform_and_independent_across_groups(oracle):
    n = 20000
    a = np.array([oracle.tail_word(9, 4, 2, 11, 0, i) for i in range(n)], dtype=np.float64) / 2.0**32
    b = np.array([oracle.tail_word(9, 4, 2, 11, 1, i) for i in range(n)], dtype=np.float64) / 2.0**32
    from scipy import stats
    assert stats.kstest(a, "uniform").pvalue > 1e-4 and stats.kstest(b, "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / np.sqrt(n)
    # joint uniformity of the leading nibbles of the two streams at equal indices
    ha, hb = (a * 16).astype(int), (b * 16).astype(int)
    assert _joint_g_test(ha, hb, 16)[2] > P_MIN
