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
