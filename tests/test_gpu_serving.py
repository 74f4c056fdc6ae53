"""Serving on the GPU: jobs that arrive while others run join the batch, and
every job's streamed W^2(t) equals, exactly, the same job run alone."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_1705_01022_gb300 as g
    g.build()
    return g


def test_each_result_is_the_same_alone_and_in_the_mix(g):
    from paper_1705_01022_gb300 import _lib, serve
    jobs = serve.poisson_jobs(14, rate=400.0, master_seed=5, L_range=(128, 1024),
                              t_range=(5, 60), seed_fn=_lib.oct_replica_seed)
    # a budget that holds only part of the jobs at a time forces staggered admission
    budget = 3 * serve.footprint(1024)
    streamed = []
    eng = serve.ServingEngine(budget, max_chunk=8, on_result=lambda j, r: streamed.append((j.jid, r)))
    done = eng.run(jobs)
    assert len(done) == len(jobs) and eng.used == 0
    assert len(streamed) == sum(len(j.measure_at) for j in jobs)
    for job in done:
        assert job.shape != (0, 0)
        with g.Simulation(job.L, job.p, job.q, job.seed, Bx=job.shape[0], By=job.shape[1]) as sim:
            t = 0
            for (tt, s1, s2, w2, net) in job.results:
                sim.run(tt - t)
                t = tt
                m = sim.measure()
                assert (tt, s1, s2, w2, net) == (m.t, m.s1, m.s2, m.w2, m.net_flips), job.jid
    # work of different jobs overlapped: some job was admitted before another finished
    by_adm = sorted(done, key=lambda j: j.admitted)
    assert any(b.admitted < a.done for a, b in zip(by_adm, by_adm[1:]))
    s = serve.summary(done, max(j.done for j in done) - min(j.arrival for j in done))
    assert s["p50_latency_s"] > 0


def test_full_warp_jobs_in_the_mix(g):
    """A job whose lattice takes full-warp sub-tiles under the 'large' policy
    (L = 8192: 1024 x 16) shares the batch with packed small jobs; every
    streamed W^2 equals the job run alone on the same sub-tile."""
    from paper_1705_01022_gb300 import _lib, serve
    from paper_1705_01022_gb300.autotune import batch_shape
    assert batch_shape(8192, "large") == (1024, 16)
    jobs = [serve.Job(0, 8192, 0.95, 0.05, _lib.oct_replica_seed(8, 0), 6, arrival=0.0,
                      measure_at=serve.log_times(6, 3)),
            serve.Job(1, 256, 1.0, 0.0, _lib.oct_replica_seed(8, 1), 9, arrival=0.0,
                      measure_at=serve.log_times(9, 4)),
            serve.Job(2, 384, 0.5, 0.5, _lib.oct_replica_seed(8, 2), 4, arrival=0.0,
                      measure_at=serve.log_times(4, 3))]
    eng = serve.ServingEngine(1 << 30, max_chunk=4)
    done = eng.run(jobs)
    assert {j.jid for j in done} == {0, 1, 2}
    for job in done:
        assert job.shape == batch_shape(job.L, "large")
        with g.Simulation(job.L, job.p, job.q, job.seed, Bx=job.shape[0], By=job.shape[1]) as sim:
            t = 0
            for (tt, s1, s2, w2, net) in job.results:
                sim.run(tt - t)
                t = tt
                m = sim.measure()
                assert (tt, s1, s2, w2, net) == (m.t, m.s1, m.s2, m.w2, m.net_flips), job.jid


def test_stream_marks(g):
    """oct_batch_mark / _done / _wait: a mark is passed once the device has run
    the MCS enqueued before it; marks not handed out are refused; a mark more
    than 64 marks old reads as passed."""
    from paper_1705_01022_gb300 import _lib
    r = _lib.oct_replica()
    r.L, r.p, r.q, r.seed = 1024, 0.95, 0.05, 3
    h = _lib.oct_batch_create([r], None)
    try:
        _lib.oct_batch_run(h, 3)
        m = _lib.oct_batch_mark(h)
        _lib.oct_batch_mark_wait(h, m)
        assert _lib.oct_batch_mark_done(h, m)
        for bad in (-1, m + 1):
            with pytest.raises(_lib.OctError):
                _lib.oct_batch_mark_done(h, bad)
            with pytest.raises(_lib.OctError):
                _lib.oct_batch_mark_wait(h, bad)
        marks = []
        for _ in range(70):
            _lib.oct_batch_run(h, 1)
            marks.append(_lib.oct_batch_mark(h))
        assert _lib.oct_batch_mark_done(h, marks[0])  # recycled: passed before its event was reused
        _lib.oct_batch_mark_wait(h, marks[-1])
        assert all(_lib.oct_batch_mark_done(h, x) for x in marks)
    finally:
        _lib.oct_batch_destroy(h)
