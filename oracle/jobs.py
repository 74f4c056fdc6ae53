"""Picklable oracle jobs for process pools (test infrastructure).

Pools that run these must use the "spawn" start method (or start before the
parent touches the GPU)."""
from __future__ import annotations


def dtrdt_final_canonical(args):
    """O2 from the flat start: returns (canonical words, net flips, (S1, S2))."""
    import oracle
    L, p, q, seed, Bx, By, n = args
    X, Y = oracle.flat(L)
    net = oracle.dtrdt_run(X, Y, oracle.Params(L=L, p=p, q=q, seed=seed, Bx=Bx, By=By), 0, n)[0]
    s1, s2, _ = oracle.w2_sums(X, Y)
    return oracle.pack_canonical(X, Y), net, (s1, s2)


def window_mcs(args):
    """O2 for MCS t on a window (rows, columns) whose corner is global site
    (wx, wy); returns the window's interior rows [y0, y1) and columns [x0, x1)
    after the MCS."""
    import oracle
    prm, t, wx, wy, Xw, Yw, (y0, y1, x0, x1) = args
    Xw, Yw = Xw.copy(), Yw.copy()
    oracle.dtrdt_mcs_window(Xw, Yw, oracle.Params(**prm), t, wx, wy)
    return Xw[y0:y1, x0:x1].copy(), Yw[y0:y1, x0:x1].copy()


def dtrdt_final_canonical_cells(args):
    """O2 from the flat start with a thread cell (cx, cy): (canonical words, net flips, (S1, S2))."""
    import oracle
    L, p, q, seed, Bx, By, cx, cy, n = args
    X, Y = oracle.flat(L)
    prm = oracle.Params(L=L, p=p, q=q, seed=seed, Bx=Bx, By=By, cx=cx, cy=cy)
    net = oracle.dtrdt_run(X, Y, prm, 0, n)[0]
    s1, s2, _ = oracle.w2_sums(X, Y)
    return oracle.pack_canonical(X, Y), net, (s1, s2)
