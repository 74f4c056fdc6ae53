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
