"""GPU two-time autocorrelations (Sec. 2: C_h, C_s of Eq. (5)) against the
oracle, through the C ABI.

Bar: the integer sums (sum h(t), sum h(s), sum h(t) h(s), the occupation
counts) are equal integers and C_h, C_s the same doubles.  The row pass takes
rows in chunks of 256 words (8 per lane); sizes cover the scalar load path
(rows of 6, 130 and 258 words), the 16-byte path (8, 132, 256 and 260 words),
partial chunks alone and after a full one, and a bare-buffer call at L = 96.  At L = 2^17 (the bench size) the oracle
cannot integrate 1.7e10 sites in a test, so properties that hold at any size
are checked there: C_h(s,s) = W^2(s) exactly, C_s(s,s) = 1/4, symmetry in
(t, s) and Cauchy-Schwarz."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def _bits(g, sim):
    return g.planes_to_bits(sim.planes(), sim.L)


def _assert_ac_equal(ac, ref, what=""):
    assert (ac.sum_ht, ac.sum_hs, ac.cross) == (ref["sum_ht"], ref["sum_hs"], ref["cross"]), what
    assert (ac.occ_x, ac.occ_y, ac.m_t, ac.m_s) == (ref["occ_x"], ref["occ_y"], ref["m_t"], ref["m_s"]), what
    assert ac.c_h == ref["c_h"] and ac.c_s == ref["c_s"], what


@pytest.mark.parametrize("L,p,q,s,dt", [
    (256, 1.0, 0.0, 3, 10),      # 8 words per row, vector path, one chunk
    (192, 0.95, 0.05, 2, 5),     # 6 words per row: scalar path
    (4160, 0.5, 0.5, 2, 3),      # 130 words: scalar path, ragged second chunk
    (4224, 1.0, 0.0, 4, 2),      # 132 words: vector path, ragged second chunk
    (8192, 0.95, 0.05, 1, 1),    # 256 words: vector path, one full chunk
    (8256, 0.5, 0.5, 2, 1),      # 258 words: scalar path, a full chunk and a ragged one of 2 words
    (8320, 0.95, 0.05, 1, 2),    # 260 words: vector path, a full chunk and a ragged one of 4 words
])
def test_handle_against_oracle(g, oracle, L, p, q, s, dt):
    Bx, By = (64, 64) if L % 128 == 0 else (32, 32)
    with g.Simulation(L, p, q, 11, Bx=Bx, By=By) as sim:
        sim.run(s)
        sim.snapshot()
        Xs, Ys = _bits(g, sim)
        ac0 = sim.measure_ac()
        _assert_ac_equal(ac0, oracle.two_time(Xs, Ys, Xs, Ys), f"L={L} t=s")
        m = sim.measure()
        assert ac0.cross == m.s2 and ac0.c_h == m.w2 and ac0.c_s == 0.25
        sim.run(dt)
        Xt, Yt = _bits(g, sim)
        ac = sim.measure_ac()
        assert (ac.t, ac.s) == (s + dt, s)
        _assert_ac_equal(ac, oracle.two_time(Xt, Yt, Xs, Ys), f"L={L}")


def test_snapshot_required(g):
    with g.Simulation(64, 1.0, 0.0, 1) as sim:
        with pytest.raises(g.OctError):
            sim.measure_ac()


def test_bare_buffers_at_L96(g, oracle):
    import torch
    from oracle import Params
    L = 96
    Xs, Ys = oracle.flat(L)
    oracle.dtrdt_run(Xs, Ys, Params(L=L, p=0.95, q=0.05, seed=3, Bx=8, By=8), 0, 4)
    Xt, Yt = Xs.copy(), Ys.copy()
    oracle.dtrdt_run(Xt, Yt, Params(L=L, p=0.95, q=0.05, seed=3, Bx=8, By=8), 4, 6)
    lt = torch.from_numpy(oracle.pack_planar(Xt, Yt).view(np.int32)).cuda()
    ls = torch.from_numpy(oracle.pack_planar(Xs, Ys).view(np.int32)).cuda()
    ac = g.two_time(lt, ls, L)
    assert (ac.t, ac.s) == (-1, -1)
    _assert_ac_equal(ac, oracle.two_time(Xt, Yt, Xs, Ys), "L=96 bare")
    # unaligned buffers take the scalar path and give the same sums
    big_t = torch.zeros(lt.numel() + 1, dtype=torch.int32, device="cuda")
    big_s = torch.zeros(ls.numel() + 1, dtype=torch.int32, device="cuda")
    big_t[1:] = lt
    big_s[1:] = ls
    ac2 = g.two_time(big_t[1:], big_s[1:], L)
    _assert_ac_equal(ac2, oracle.two_time(Xt, Yt, Xs, Ys), "L=96 unaligned")


def test_full_size_properties(g):
    import torch
    L = 1 << 17
    # one stream for the handle, the copy and the bare-buffer calls: the
    # library's own streams do not synchronise with torch's default stream
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        lat = torch.empty(L * L // 16, dtype=torch.int32, device="cuda")
        with g.Simulation(L, 0.95, 0.05, 1, Bx=256, By=64, stream=st, lattice=lat) as sim:
            sim.run(2)
            sim.snapshot()
            m = sim.measure()
            ac = sim.measure_ac()
            assert ac.cross == m.s2 and ac.sum_ht == m.s1 and ac.c_h == m.w2
            assert ac.c_s == 0.25 and ac.m_t == ac.m_s == L * L
            snap = lat.clone()
            sim.run(1)
            m1 = sim.measure()
            a = g.two_time(lat, snap, L, stream=st)
            b = g.two_time(snap, lat, L, stream=st)
            assert (a.cross, a.sum_ht, a.sum_hs) == (b.cross, b.sum_hs, b.sum_ht)
            assert a.c_h == b.c_h and a.c_s == b.c_s
            assert a.sum_ht == m1.s1 and a.sum_hs == m.s1
            ac1 = sim.measure_ac()
            assert (ac1.cross, ac1.c_h, ac1.c_s) == (a.cross, a.c_h, a.c_s)
            assert (ac1.occ_x, ac1.occ_y) == (a.occ_x, a.occ_y)
            assert 0.0 < a.c_h and a.c_h ** 2 <= m1.w2 * m.w2
            assert 0.0 < a.c_s < 0.25
        del snap
    st.synchronize()
