"""Asynchronous measurement and read-back through the C ABI
(oct_measure_w2_async / oct_w2_wait, oct_get_planes_async): the results equal
the synchronous calls' and the oracle's, work enqueued after an asynchronous
measurement does not change it, misuse is rejected, and two handles driven
in an interleaved pipeline from one host thread (the end-to-end loop of the
benchmark, with page-locked host buffers) follow the oracle bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def _oracle_after(oracle, L, p, q, seed, Bx, By, planes, t0, n):
    from oracle import Params
    X, Y = _bits(L, planes)
    oracle.dtrdt_run(X, Y, Params(L=L, p=p, q=q, seed=seed, Bx=Bx, By=By), t0, n)
    return X, Y


def _bits(L, planes):
    import paper_1705_01022_gb300 as g
    return g.planes_to_bits(planes, L)


def test_async_measure_is_the_lattice_at_enqueue_time(g, oracle):
    from paper_1705_01022_gb300 import _lib
    L, p, q, seed = 256, 0.95, 0.05, 31
    with g.Simulation(L, p, q, seed, Bx=64, By=64) as sim:
        sim.run(3)
        ref = sim.measure()
        sim.measure_async()
        with pytest.raises(_lib.OctError) as e:
            sim.measure_async()
        assert e.value.code == _lib.OCT_EINVAL
        with pytest.raises(_lib.OctError):
            sim.measure()
        sim.run(2)  # enqueued after the measurement
        w = sim.w2_wait()
        assert (w.t, w.s1, w.s2, w.w2, w.net_flips) == (3, ref.s1, ref.s2, ref.w2, ref.net_flips)
        with pytest.raises(_lib.OctError):
            sim.w2_wait()
        m5 = sim.measure()
        assert m5.t == 5
        X, Y = _bits(L, sim.planes())
        s1, s2, _ = oracle.w2_sums(X, Y)
        assert (m5.s1, m5.s2, m5.w2) == (s1, s2, oracle.w2(X, Y))


def test_async_planes_match_sync(g):
    from paper_1705_01022_gb300 import _lib
    L = 512
    with g.Simulation(L, 0.7, 0.3, 5, Bx=128, By=64) as sim:
        sim.run(2)
        buf = np.zeros(L * L // 16, np.uint32)
        _lib.oct_get_planes_async(sim.h, buf, buf.size)
        sim.sync()
        assert np.array_equal(buf, sim.planes())
        with pytest.raises(_lib.OctError):
            _lib.oct_get_planes_async(sim.h, buf, buf.size - 1)


def test_interleaved_pipeline_of_two_handles(g, oracle):
    import torch
    from paper_1705_01022_gb300 import _lib
    L, p, q, Bx, By = 1024, 0.95, 0.05, 256, 64
    seeds = (41, 42)
    words = L * L // 16
    sims = [g.Simulation(L, p, q, s, Bx=Bx, By=By) for s in seeds]
    try:
        for s in sims:
            s.run(1)
        start = [s.planes() for s in sims]
        hosts = [torch.from_numpy(w.view(np.int32).copy()).pin_memory() for w in start]
        pending = [False, False]
        results = [[], []]
        for i in range(6):  # three steps per handle, one MCS each, interleaved
            k = i % 2
            h = sims[k].h
            if pending[k]:
                results[k].append(_lib.oct_w2_wait(h))
            _lib.oct_set_planes(h, hosts[k].data_ptr(), words, 1 + i // 2)
            _lib.oct_run_mcs(h, 1)
            _lib.oct_measure_w2_async(h)
            _lib.oct_get_planes_async(h, hosts[k].data_ptr(), words)
            pending[k] = True
        for k in range(2):
            results[k].append(_lib.oct_w2_wait(sims[k].h))
        for k, seed in enumerate(seeds):
            X, Y = _bits(L, start[k])
            for n, w in enumerate(results[k]):
                from oracle import Params
                oracle.dtrdt_run(X, Y, Params(L=L, p=p, q=q, seed=seed, Bx=Bx, By=By), 1 + n, 1)
                s1, s2, _ = oracle.w2_sums(X, Y)
                assert (w.t, w.s1, w.s2, w.w2) == (2 + n, s1, s2, oracle.w2(X, Y)), (k, n)
            Xh, Yh = _bits(L, hosts[k].numpy().view(np.uint32))
            assert np.array_equal(Xh, X) and np.array_equal(Yh, Y)
    finally:
        for s in sims:
            s.close()
