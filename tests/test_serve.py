"""Host logic of the continuous-batching serving loop (no GPU): admission by
memory budget, first-come-first-served order, measurement times, slot reuse
and latency bookkeeping, driven by a fake batch on a virtual clock."""
import math

import pytest

from paper_1705_01022_gb300 import serve


class VirtualClock:
    def __init__(self):
        self.now = 0.0

    def __call__(self):
        return self.now

    def advance_to(self, t):
        self.now = max(self.now, t)


class FakeBatch:
    """Keeps per-slot times; time passes in proportion to the work run."""

    def __init__(self, clock, rate=1e6):
        self.clock, self.rate = clock, rate
        self.slots, self.t, self.free, self.max_slots = {}, {}, [], 0
        self.runs = []

    def add(self, job):
        slot = self.free.pop() if self.free else len(self.t)
        self.slots[slot] = job
        self.t[slot] = 0
        self.max_slots = max(self.max_slots, len(self.slots))
        return slot

    def remove(self, slot):
        del self.slots[slot]
        self.free.append(slot)

    def run(self, n):
        work = sum(j.L * j.L for j in self.slots.values()) * n
        for s in self.slots:
            self.t[s] += n
        self.runs.append((n, len(self.slots)))
        self.clock.now += work / self.rate

    def measure(self, slot):
        job = self.slots[slot]
        return (self.t[slot], job.jid, 0, float(self.t[slot]), 0)


def test_log_times():
    for t_max in (1, 2, 10, 37, 10_000):
        ts = serve.log_times(t_max)
        assert ts[0] == 1 and ts[-1] == t_max
        assert all(b > a for a, b in zip(ts, ts[1:]))


def test_poisson_jobs_follow_the_recipe():
    jobs = serve.poisson_jobs(400, rate=10.0, master_seed=3)
    arr = [j.arrival for j in jobs]
    assert all(b >= a for a, b in zip(arr, arr[1:]))
    assert all(j.L % 128 == 0 and 128 <= j.L <= 16384 for j in jobs)
    assert all(10 <= j.t_max <= 10_000 for j in jobs)
    assert {(j.p, j.q) for j in jobs} == set(serve.PQ_SET)
    # log-uniform L: about half the jobs below the geometric mean of the range
    below = sum(j.L < math.sqrt(128 * 16384) for j in jobs) / len(jobs)
    assert 0.4 < below < 0.6
    mean_gap = (arr[-1] - arr[0]) / (len(arr) - 1)
    assert 0.08 < mean_gap < 0.12


def test_engine_respects_budget_order_and_measurement_times():
    clock = VirtualClock()
    fb = FakeBatch(clock)
    budget = 3 * serve.footprint(1024)
    eng = serve.ServingEngine(budget, batch=fb, max_chunk=16, clock=clock)
    seen = []
    eng.on_result = lambda job, res: seen.append((job.jid, res[0]))
    jobs = [serve.Job(i, 1024 if i % 2 else 512, 1.0, 0.0, i, t_max=20 + 7 * i,
                      arrival=0.5 * i, measure_at=serve.log_times(20 + 7 * i)) for i in range(8)]
    done = eng.run(jobs, realtime=False)
    assert len(done) == 8
    assert eng.used == 0 and not eng.running
    for j in done:
        assert [r[0] for r in j.results] == j.measure_at
        assert j.admitted >= j.arrival and j.done >= j.admitted
    # budget never exceeded: at most 3 jobs of 1024 worth of memory at once
    assert fb.max_slots <= 6
    assert max(k for _, k in fb.runs) <= 6
    # first come, first served
    adm = sorted(done, key=lambda j: j.admitted)
    assert [j.jid for j in adm] == sorted(j.jid for j in adm)
    # slots are reused
    assert len(fb.t) < len(jobs)
    assert len(seen) == sum(len(j.measure_at) for j in jobs)
    s = serve.summary(done, clock.now)
    assert s["jobs"] == 8 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_engine_rejects_jobs_larger_than_the_budget():
    eng = serve.ServingEngine(1000, batch=FakeBatch(VirtualClock()))
    with pytest.raises(ValueError):
        eng.submit(serve.Job(0, 1024, 1.0, 0.0, 1, t_max=10))


def _jobs(n):
    return [serve.Job(i, 128, 1.0, 0.0, 1000 + i, 20, arrival=0.0, measure_at=serve.log_times(20, 4))
            for i in range(n)]


def test_cancel_waiting_and_running_jobs():
    clock = VirtualClock()
    fb = FakeBatch(clock)
    eng = serve.ServingEngine(hbm_budget=2 * serve.footprint(128), batch=fb, clock=clock)
    jobs = _jobs(4)
    for j in jobs:
        eng.submit(j)
    eng.tick(0.0)  # admits two (the budget holds two lattices), runs them to their first event
    assert len(eng.running) == 2 and len(eng.waiting) == 2
    assert eng.cancel(3)                      # waiting: leaves the queue
    assert eng.cancel(0)                      # running: leaves the batch, memory back
    assert not eng.cancel(0) and not eng.cancel(99)
    assert eng.used == serve.footprint(128) and 0 not in [j.jid for j in eng.running.values()]
    while eng.waiting or eng.running:
        eng.tick(clock())
    done = sorted(j.jid for j in eng.finished)
    assert done == [1, 2]
    assert jobs[0].cancelled and jobs[3].cancelled and not jobs[1].cancelled
    assert jobs[0].results and not jobs[3].results  # what was streamed before the cancel stays


def test_admission_budget_of_zero_rejects_everything():
    eng = serve.ServingEngine(hbm_budget=0, batch=FakeBatch(VirtualClock()), clock=VirtualClock())
    with pytest.raises(ValueError):
        eng.submit(_jobs(1)[0])


def test_jsonl_metrics_lines():
    import io
    import json
    clock = VirtualClock()
    buf = io.StringIO()
    eng = serve.ServingEngine(hbm_budget=10 * serve.footprint(128), batch=FakeBatch(clock), clock=clock,
                              on_result=serve.jsonl_logger(buf, clock))
    jobs = _jobs(2)
    eng.run(jobs, realtime=False)
    lines = [json.loads(x) for x in buf.getvalue().splitlines()]
    assert len(lines) == sum(len(j.measure_at) for j in jobs)
    for rec in lines:
        assert set(rec) == {"job", "L", "p", "q", "t", "s1", "s2", "n_sites", "w2", "net_flips", "since_arrival_s"}
        assert rec["n_sites"] == 128 * 128 and rec["since_arrival_s"] >= 0
    assert [r["t"] for r in lines if r["job"] == 0] == jobs[0].measure_at


class FakeAsyncBatch(FakeBatch):
    """Measures asynchronously: a measurement enqueued before a run completes
    only once that later run has been issued (like a reduction queued behind
    the MCS on one stream); a slot may be removed while its measurement is in
    flight."""

    def __init__(self, clock, rate=1e6):
        super().__init__(clock, rate)
        self.queue = []  # [result, runs issued when enqueued]

    def measure_async(self, slot):
        self.queue.append([self.measure(slot), len(self.runs)])
        return len(self.queue) - 1

    def poll(self, ticket):
        res, at = self.queue[ticket]
        return res if len(self.runs) > at else None

    def wait(self, ticket):
        return self.queue[ticket][0]


def test_asynchronous_measurements_are_all_delivered_in_order():
    clock = VirtualClock()
    fb = FakeAsyncBatch(clock)
    eng = serve.ServingEngine(3 * serve.footprint(1024), batch=fb, max_chunk=16, clock=clock)
    assert eng.async_measure
    jobs = [serve.Job(i, 1024 if i % 2 else 512, 1.0, 0.0, i, t_max=20 + 7 * i,
                      arrival=0.5 * i, measure_at=serve.log_times(20 + 7 * i)) for i in range(8)]
    done = eng.run(jobs, realtime=False)
    assert len(done) == 8 and not eng.pending and eng.used == 0
    for j in done:
        assert [r[0] for r in j.results] == j.measure_at
        assert j.done >= j.admitted >= j.arrival
    # the host never waited on a measurement while jobs were still running
    assert len(fb.queue) == sum(len(j.measure_at) for j in jobs)


class FakeMarkedBatch(FakeAsyncBatch):
    """Runs are only issued, not done: the device is a queue of issued runs
    that finishes one run per wait; marks record the issued count."""

    def __init__(self, clock, rate=1e6):
        super().__init__(clock, rate)
        self.marks, self.done_runs, self.max_ahead, self.last_waited = [], 0, 0, -1

    def run(self, n):
        super().run(n)
        self.max_ahead = max(self.max_ahead, len(self.runs) - self.done_runs)

    def mark(self):
        self.marks.append(len(self.runs))
        return len(self.marks) - 1

    def mark_done(self, m):
        return self.marks[m] <= self.done_runs

    def wait_mark(self, m):
        assert m > self.last_waited  # oldest first
        self.last_waited = m
        self.done_runs = max(self.done_runs, self.marks[m])


@pytest.mark.parametrize("max_inflight", [1, 2, 4])
def test_engine_keeps_at_most_max_inflight_ticks_ahead(max_inflight):
    """With stream marks, the host waits for the tick max_inflight ticks back
    before it goes on, so a newly admitted job joins launches that follow at
    most max_inflight enqueued ticks; every job still gets all its results."""
    clock = VirtualClock()
    fb = FakeMarkedBatch(clock)
    eng = serve.ServingEngine(4 * serve.footprint(1024), batch=fb, max_chunk=8, clock=clock,
                              max_inflight=max_inflight)
    assert eng.throttled
    jobs = [serve.Job(i, 512 + 128 * (i % 4), 1.0, 0.0, i, t_max=30 + 11 * i,
                      arrival=0.3 * i, measure_at=serve.log_times(30 + 11 * i)) for i in range(10)]
    done = eng.run(jobs, realtime=False)
    assert len(done) == 10 and not eng.pending and eng.used == 0
    for j in done:
        assert [r[0] for r in j.results] == j.measure_at
    assert len(fb.marks) == eng.ticks
    # after each tick at most max_inflight ticks were issued and not yet passed
    assert fb.max_ahead <= max_inflight
    assert len(eng.inflight[0]) <= max_inflight


def test_jobs_spread_over_several_batches_that_tick_independently():
    """With two batches a new job joins the one with fewer running sites;
    each batch advances by its own chunks, and every job still gets all its
    measurements, in order, with the memory returned at the end."""
    clock = VirtualClock()
    fbs = [FakeMarkedBatch(clock), FakeMarkedBatch(clock)]
    eng = serve.ServingEngine(6 * serve.footprint(1024), batch=fbs, max_chunk=8, clock=clock, max_inflight=2)
    jobs = [serve.Job(i, [1024, 256, 512, 768][i % 4], 1.0, 0.0, i, t_max=25 + 13 * i,
                      arrival=0.2 * i, measure_at=serve.log_times(25 + 13 * i)) for i in range(12)]
    done = eng.run(jobs, realtime=False)
    assert len(done) == 12 and not eng.pending and not eng.running and eng.used == 0
    for j in done:
        assert j.batch in (0, 1)
        assert [r[0] for r in j.results] == j.measure_at
    used = {j.batch for j in done}
    assert used == {0, 1}
    # the batches ran different chunk sequences (they do not move in lock step)
    assert [n for n, _ in fbs[0].runs] != [n for n, _ in fbs[1].runs]
    # the first two jobs (both arriving while nothing runs) went to different batches
    assert jobs[0].batch != jobs[1].batch


def test_cancel_with_several_batches():
    """A running job leaves the batch it runs in (the engine keys running jobs
    by batch and slot, and two batches hand out the same slot numbers); the
    jobs of the other batch keep running to their end."""
    clock = VirtualClock()
    fbs = [FakeBatch(clock), FakeBatch(clock)]
    eng = serve.ServingEngine(hbm_budget=4 * serve.footprint(128), batch=fbs, clock=clock)
    jobs = _jobs(4)
    for j in jobs:
        eng.submit(j)
    eng.tick(0.0)
    assert {j.batch for j in eng.running.values()} == {0, 1}
    # slot 0 exists in both batches: cancelling job 1 must remove only its own replica
    b1, s1 = jobs[1].batch, jobs[1].slot
    other = [j for j in jobs if j.jid != 1 and (j.batch, j.slot) != (b1, s1)]
    assert any(j.slot == s1 for j in other)
    assert eng.cancel(1)
    assert s1 not in fbs[b1].slots and all(j.slot in fbs[j.batch].slots for j in other if j in eng.running.values())
    while eng.waiting or eng.running:
        eng.tick(clock())
    assert sorted(j.jid for j in eng.finished) == [0, 2, 3] and eng.used == 0
    for j in eng.finished:
        assert [r[0] for r in j.results] == j.measure_at
