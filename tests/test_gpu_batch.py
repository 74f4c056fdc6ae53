"""Batched replicas: every replica of a batch equals, bit for bit, the same
realization run alone through the plain entry points (and so the oracle), for
mixed L, p, q and sub-tile shapes; graph replay and launch-by-launch runs agree;
replica keys match the oracle's derivation."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def test_replica_seed_matches_oracle(g, oracle):
    from paper_1705_01022_gb300 import _lib
    for master in (1, 7, 2**40 + 3, 2**64 - 1):
        for r in (0, 1, 2, 1000, 2047, 2**31):
            assert _lib.oct_replica_seed(master, r) == oracle.replica_seed(master, r)


PQ = [(1.0, 0.0), (0.95, 0.05), (0.5, 0.5)]


def _replicas(g, master=7):
    from paper_1705_01022_gb300 import _lib
    reps = []
    Ls = [64, 128, 192, 256, 320, 384, 448, 512]
    for i, L in enumerate(Ls):
        for j, (p, q) in enumerate(PQ):
            r = len(reps)
            reps.append((L, p, q, _lib.oct_replica_seed(master, r)))
    # explicit shapes too: a full-warp sub-tile and a two-group one
    reps.append((1024, 0.95, 0.05, 99, 256, 64))
    reps.append((512, 0.5, 0.5, 98, 64, 32))
    # full-warp sub-tiles of both acceptance modes (the uniform-row-offset kernel)
    reps.append((1024, 1.0, 0.0, 97, 512, 32))
    reps.append((512, 0.6, 0.3, 96, 128, 128))
    return reps


def test_batch_equals_plain_runs(g):
    reps = _replicas(g)
    n = 5
    with g.Batch(reps) as b:
        b.run(n)
        res = b.measure()
        for i, r in enumerate(reps):
            L, p, q, seed = r[:4]
            Bx, By = (r[4], r[5]) if len(r) > 4 else ((64, 64) if L % 128 == 0 else (32, 32))
            with g.Simulation(L, p, q, seed, Bx=Bx, By=By) as sim:
                sim.run(n)
                assert np.array_equal(b.planes(i), sim.planes()), (i, r)
                m = sim.measure()
                assert (res[i].s1, res[i].s2, res[i].hmax, res[i].net_flips) == \
                    (m.s1, m.s2, m.hmax, m.net_flips), (i, r)
                assert res[i].w2 == m.w2


def test_batch_matches_oracle(g, oracle):
    reps = [(192, 0.95, 0.05, 5), (256, 0.5, 0.5, 6), (64, 1.0, 0.0, 7)]
    with g.Batch(reps) as b:
        b.run(4)
        for i, (L, p, q, seed) in enumerate(reps):
            B = 64 if L % 128 == 0 else 32
            X, Y = oracle.flat(L)
            oracle.dtrdt_run(X, Y, oracle.Params(L=L, p=p, q=q, seed=seed, Bx=B, By=B), 0, 4)
            assert np.array_equal(b.planes(i), oracle.pack_planar(X, Y)), i


def test_kinds_split_into_parts_equal_plain_runs(g):
    """Replica sets large enough that the batch splits a kind into several
    parts (each at least 2^26 sites, at most three; each part a branch of the
    captured graph): 13 full-warp replicas of L = 4096 with both rates random
    (218 M sites: three parts), 9 of L = 4096 in KPZ (151 M: two parts), and
    packed one-group-wide replicas of L = 3968 (one part).  Five MCS run as one
    four-MCS graph and one single MCS; every replica equals its plain run."""
    from paper_1705_01022_gb300 import _lib
    from paper_1705_01022_gb300.autotune import batch_shape
    reps = []
    for i in range(13):
        reps.append((4096, 0.95, 0.05, _lib.oct_replica_seed(21, i)))
    for i in range(9):
        reps.append((4096, 1.0, 0.0, _lib.oct_replica_seed(22, i)))
    for i in range(4):
        reps.append((3968, 0.5, 0.5, _lib.oct_replica_seed(23, i)))
    reps = [r + batch_shape(r[0], "tall") for r in reps]
    assert reps[0][4:] == (1024, 16) and reps[-1][4:] == (32, 64)
    n = 5
    with g.Batch(reps) as b:
        b.run(n)
        res = b.measure()
        for i, r in enumerate(reps):
            L, p, q, seed, Bx, By = r
            with g.Simulation(L, p, q, seed, Bx=Bx, By=By) as sim:
                sim.run(n)
                assert np.array_equal(b.planes(i), sim.planes()), (i, r)
                m = sim.measure()
                assert (res[i].t, res[i].s1, res[i].s2, res[i].net_flips) == (n, m.s1, m.s2, m.net_flips), (i, r)


def test_graph_and_timed_launches_agree(g):
    from paper_1705_01022_gb300 import _lib
    reps = _replicas(g, master=11)[:12]
    with g.Batch(reps) as a, g.Batch(reps) as b:
        a.run(3)
        _lib.oct_batch_set_timing(b.h, True)
        b.run(3)
        ms, launches = _lib.oct_batch_get_timing(b.h)
        assert launches == 12 and ms > 0
        for i in range(len(reps)):
            assert np.array_equal(a.planes(i), b.planes(i))
        t, n, sites, draws = a.stats()
        assert (t, n) == (3, len(reps))
        assert sites == sum(r[0] * r[0] for r in reps)


def test_invalid_replicas_rejected(g):
    from paper_1705_01022_gb300 import _lib
    with pytest.raises(_lib.OctError):
        g.Batch([(100, 1.0, 0.0, 1)])
    with pytest.raises(_lib.OctError):
        g.Batch([(256, 1.0, 0.0, 1, 96, 32)])


def test_async_measurements_equal_sync_ones(g):
    """oct_batch_measure_async behind the batch's MCS equals the synchronous
    measurement of the same state, also when the replica is removed (and its
    slot reused) right after the call and when membership changes between
    runs (the work list is rebuilt without waiting for the device)."""
    from paper_1705_01022_gb300 import _lib
    reps = _replicas(g, master=13)[:10]
    with g.Batch(reps) as b, g.Batch(reps) as ref:
        tickets = []
        for rnd in range(3):
            b.run(2)
            ref.run(2)
            for slot in range(len(reps)):
                if rnd < 2 or slot % 2 == 0:
                    tickets.append((rnd, slot, _lib.oct_batch_measure_async(b.h, slot)))
            want = {slot: _lib.oct_batch_measure_slot(ref.h, slot) for slot in range(len(reps))
                    if rnd < 2 or slot % 2 == 0}
            for r_, slot, tk in tickets:
                if r_ != rnd:
                    continue
                got = _lib.oct_batch_wait(b.h, tk)
                w = want[slot]
                assert (got.t, got.s1, got.s2, got.hmax, got.net_flips, got.w2) == \
                    (w.t, w.s1, w.s2, w.hmax, w.net_flips, w.w2), (rnd, slot)
            if rnd == 1:
                # odd slots leave right after their measurement; one new replica joins each batch
                for slot in range(1, len(reps), 2):
                    _lib.oct_batch_remove(b.h, slot)
                    _lib.oct_batch_remove(ref.h, slot)
                extra = _lib.oct_replica()
                extra.L, extra.p, extra.q, extra.seed = 256, 0.95, 0.05, 4242
                assert _lib.oct_batch_add(b.h, extra) == _lib.oct_batch_add(ref.h, extra)
        got = _lib.oct_batch_poll(b.h, tickets[-1][2])
        assert got is not None  # long done: poll reports it ready
        with pytest.raises(_lib.OctError):
            _lib.oct_batch_poll(b.h, 10**6)
