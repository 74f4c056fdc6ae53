"""Continuous-batching serving loop for octahedron-model simulation jobs.

A job is one realization (L, p, q, seed) to run for t_max MCS, with W^2 sent
back at log-spaced times.  Jobs arrive over time (e.g. as a Poisson stream).
The engine keeps one or more batches (``oct_batch_*`` in include/oct.h), each
on its own stream, whose replicas are the running jobs, each on the sub-tile
its shape policy gives (see autotune.batch_shape; the shape is recorded in the
job, since it is part of the job's dynamics):

* admission: a waiting job that has arrived joins the batch as soon as its
  lattice fits the HBM budget (first come, first served);
* a tick of a batch advances all its running jobs together by the same
  number of MCS (up to the next measurement or finish among them, at most
  ``max_chunk``), so work of jobs that arrived at different times overlaps on
  the device; batches tick independently (a new job joins the batch with the
  fewest running sites), so their launches overlap too;
* at a job's measurement times its exact W^2 is computed on the device and
  handed to the ``on_result`` callback (streamed back).  With a batch that
  measures asynchronously (``measure_async`` / ``poll``), the reduction is
  enqueued behind the job's MCS and the result delivered when it is done, so
  the host never waits for the device between ticks;
* a job that reaches t_max leaves the batch and returns its memory; its
  latency ends when its last result has been delivered.

Each job's trajectory is the same as running it alone: its random numbers
depend only on its own key and its own time, not on the mix.
"""
from __future__ import annotations

import bisect
import math
import time
from collections import deque
from dataclasses import dataclass, field

PQ_SET = [(1.0, 0.0), (0.8, 0.2), (0.5, 0.5)]


@dataclass
class Job:
    jid: int
    L: int
    p: float
    q: float
    seed: int
    t_max: int
    arrival: float = 0.0
    measure_at: list = field(default_factory=list)
    # set by the engine
    slot: int = -1
    t: int = 0
    admitted: float | None = None
    done: float | None = None
    results: list = field(default_factory=list)  # (t, s1, s2, w2, net_flips)
    cancelled: bool = False
    shape: tuple = (0, 0)  # sub-tile (Bx, By) the engine chose; part of the job's dynamics
    batch: int = -1        # index of the engine's batch the job runs in

    @property
    def attempts(self) -> int:
        return self.L * self.L * self.t_max

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def footprint(L: int) -> int:
    """Device bytes a job holds while running: its packed lattice."""
    return L * L // 4


def log_times(t_max: int, n: int = 8):
    """t = round(t_max^(i/(n-1))), i = 0..n-1, made strictly increasing, ending at t_max."""
    out = []
    for i in range(n):
        t = max(1, int(round(t_max ** (i / (n - 1))))) if n > 1 else t_max
        if out and t <= out[-1]:
            t = out[-1] + 1
        if t > t_max:
            break
        out.append(t)
    if not out or out[-1] != t_max:
        out.append(t_max)
    return out


def poisson_jobs(n: int, rate: float, master_seed: int = 1, L_range=(128, 16384),
                 t_range=(10, 10_000), seed_fn=None, n_measure: int = 8):
    """n jobs with exponential inter-arrival times (rate jobs/s), L log-uniform
    in L_range rounded to a multiple of 128, t_max log-uniform in t_range,
    (p, q) uniform over PQ_SET, keys from seed_fn(master_seed, jid)."""
    import numpy as np
    rng = np.random.default_rng(master_seed)
    t = 0.0
    jobs = []
    for jid in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        L = math.exp(rng.uniform(math.log(L_range[0]), math.log(L_range[1])))
        L = int(min(L_range[1], max(L_range[0], 128 * round(L / 128))))
        t_max = int(round(math.exp(rng.uniform(math.log(t_range[0]), math.log(t_range[1])))))
        p, q = PQ_SET[int(rng.integers(0, len(PQ_SET)))]
        seed = seed_fn(master_seed, jid) if seed_fn else (master_seed << 32) + jid
        jobs.append(Job(jid, L, p, q, seed, t_max, arrival=t, measure_at=log_times(t_max, n_measure)))
    return jobs


def expected_work(L_range=(128, 16384), t_range=(10, 10_000)) -> float:
    """E[L^2 * t_max] of poisson_jobs (attempts per job), ignoring rounding."""
    a, b = L_range
    eL2 = (b * b - a * a) / (2.0 * math.log(b / a))
    c, d = t_range
    et = (d - c) / math.log(d / c)
    return eL2 * et


class ServingEngine:
    """Runs jobs through one or more dynamic batches.  A batch must offer
    add(job), remove(slot), run(n) and measure(slot) -> (t, s1, s2, w2,
    net_flips); ``batch`` is one such object or a list of them, by default
    ``n_batches`` GPU batches of this package, each on its own stream.

    With several batches a new job joins the one whose running jobs hold the
    fewest sites, and each batch advances on its own: one batch's MCS does not
    wait for another's, so a batch of small or few jobs, whose device steps
    are bound by latency rather than by work, overlaps with the others on the
    device instead of setting the pace of every job."""

    def __init__(self, hbm_budget: int, batch=None, stream=None, max_chunk: int = 64,
                 on_result=None, clock=time.perf_counter, shape_policy: str = "large",
                 max_inflight: int = 4, n_batches: int = 1):
        self.budget = int(hbm_budget)
        self.shape_policy = shape_policy  # autotune.batch_shape policy for each job's sub-tile
        self.used = 0
        if batch is None:
            batch = [GpuBatch(stream if i == 0 else None) for i in range(max(1, n_batches))]
        self.batches = list(batch) if isinstance(batch, (list, tuple)) else [batch]
        self.batch = self.batches[0]
        self.max_chunk = max_chunk
        self.on_result = on_result
        self.clock = clock
        self.waiting: deque[Job] = deque()
        self.running: dict[tuple, Job] = {}  # (batch index, slot) -> job
        self.finished: list[Job] = []
        self.pending: deque = deque()  # (job, batch index, ticket) of asynchronous measurements
        self.async_measure = all(hasattr(b, "measure_async") for b in self.batches)
        self.ticks = 0
        self.mcs_attempts = 0
        # At most max_inflight ticks of a batch stay enqueued ahead of the
        # device (stream marks): a job admitted now joins the launches right
        # behind them instead of queueing behind everything the host could
        # enqueue.  A batch at its limit is skipped until its oldest tick is done.
        self.max_inflight = max_inflight
        self.inflight = [deque() for _ in self.batches]
        self.throttled = max_inflight > 0 and all(hasattr(b, "mark") for b in self.batches)

    def submit(self, job: Job) -> None:
        if footprint(job.L) > self.budget:
            raise ValueError(f"job {job.jid} needs {footprint(job.L)} B, more than the budget")
        self.waiting.append(job)

    def _sites(self, bi: int) -> int:
        return sum(j.L * j.L for (b, _), j in self.running.items() if b == bi)

    def _admit(self, now: float) -> None:
        while self.waiting and self.waiting[0].arrival <= now:
            job = self.waiting[0]
            if self.used + footprint(job.L) > self.budget:
                break  # first come, first served: later jobs wait behind it
            self.waiting.popleft()
            from .autotune import batch_shape
            job.shape = batch_shape(job.L, self.shape_policy)
            bi = min(range(len(self.batches)), key=self._sites)
            job.batch = bi
            job.slot = self.batches[bi].add(job)
            job.admitted = now
            job.t = 0
            self.used += footprint(job.L)
            self.running[(bi, job.slot)] = job

    def _chunk(self, bi: int) -> int:
        n = self.max_chunk
        for (b, _), job in self.running.items():
            if b != bi:
                continue
            i = bisect.bisect_right(job.measure_at, job.t)
            nxt = job.measure_at[i] if i < len(job.measure_at) else job.t_max
            n = min(n, nxt - job.t)
        return max(1, n)

    def _ready(self, bi: int) -> bool:
        """Whether batch bi may take another tick (its in-flight limit)."""
        q = self.inflight[bi]
        while q and len(q) >= self.max_inflight and self.batches[bi].mark_done(q[0]):
            q.popleft()
        return len(q) < self.max_inflight

    def tick(self, now: float | None = None) -> bool:
        """Admits arrived jobs and advances the running ones of every batch
        that may take a tick to their next event.  Returns False if nothing
        was running."""
        self._admit(self.clock() if now is None else now)
        if not self.running:
            return False
        busy = {b for b, _ in self.running}
        ran = False
        for bi in sorted(busy):
            if self.throttled and not self._ready(bi):
                continue
            self._tick_batch(bi, now)
            ran = True
        if self.throttled and not ran:
            # every batch is at its limit: wait for the oldest tick of one of them
            bi = min(busy, key=lambda b: self.inflight[b][0])
            self.batches[bi].wait_mark(self.inflight[bi].popleft())
        self.deliver()
        return True

    def _tick_batch(self, bi: int, now) -> None:
        batch = self.batches[bi]
        n = self._chunk(bi)
        batch.run(n)
        self.ticks += 1
        for (b, slot), job in list(self.running.items()):
            if b != bi:
                continue
            job.t += n
            self.mcs_attempts += n * job.L * job.L
            last = job.t >= job.t_max
            if job.t in job.measure_at:
                if self.async_measure:
                    self.pending.append((job, bi, batch.measure_async(slot)))
                else:
                    self._deliver_one(job, batch.measure(slot), now)
            if last:
                batch.remove(slot)
                del self.running[(bi, slot)]
                self.used -= footprint(job.L)
                if not self.async_measure or job.t_max not in job.measure_at:
                    job.done = self.clock() if now is None else now
                    self.finished.append(job)
        if self.throttled:
            self.inflight[bi].append(batch.mark())

    def _deliver_one(self, job: Job, res, now=None) -> None:
        assert res[0] in job.measure_at, (res[0], job.measure_at)
        job.results.append(res)
        if self.on_result:
            self.on_result(job, res)
        if self.async_measure and res[0] == job.t_max:
            job.done = self.clock() if now is None else now
            self.finished.append(job)

    def deliver(self, block: bool = False) -> int:
        """Hands the finished asynchronous measurements to their jobs, in the
        order they were enqueued; with block, waits for all.  Returns the
        number delivered."""
        n = 0
        while self.pending:
            job, bi, ticket = self.pending[0]
            res = self.batches[bi].wait(ticket) if block else self.batches[bi].poll(ticket)
            if res is None:
                break
            self.pending.popleft()
            self._deliver_one(job, res)
            n += 1
        return n

    def run(self, jobs, realtime: bool = True, sleep=time.sleep) -> list[Job]:
        """Serves jobs (sorted by arrival, times relative to the start).  In
        real time a job becomes visible when the clock passes its arrival."""
        t0 = self.clock()
        for job in sorted(jobs, key=lambda j: j.arrival):
            job.arrival += t0
            self.submit(job)
        while self.waiting or self.running or self.pending:
            now = self.clock()
            if not self.tick(now):
                if self.pending and not self.waiting:
                    self.deliver(block=True)
                elif self.waiting:
                    self.deliver()
                    wait = self.waiting[0].arrival - self.clock()
                    if wait > 0 and realtime:
                        sleep(min(wait, 0.05 if not self.pending else 0.001))
                    elif not realtime:
                        self.clock_skip(self.waiting[0].arrival)
        return self.finished

    def cancel(self, jid: int) -> bool:
        """Withdraws a job: a waiting one leaves the queue, a running one leaves
        its batch at once and returns its memory (its streamed results stay).
        Returns False if the job is unknown or already finished."""
        for job in list(self.waiting):
            if job.jid == jid:
                self.waiting.remove(job)
                job.cancelled = True
                return True
        for (bi, slot), job in list(self.running.items()):
            if job.jid == jid:
                self.batches[bi].remove(slot)
                del self.running[(bi, slot)]
                self.used -= footprint(job.L)
                job.cancelled = True
                return True
        return False

    def clock_skip(self, t: float) -> None:
        """Advances a virtual clock (only meaningful with an injected clock)."""
        if hasattr(self.clock, "advance_to"):
            self.clock.advance_to(t)

    def close(self) -> None:
        """Releases every batch that has a close method."""
        for b in self.batches:
            if hasattr(b, "close"):
                b.close()


def jsonl_logger(fp, clock=time.perf_counter):
    """An on_result callback writing one JSON line per streamed measurement:
    job id, L, p, q, t, S1, S2 (as integers), N, W^2, net flips, and the
    seconds since the job arrived."""
    import json

    def log(job: Job, res) -> None:
        t, s1, s2, w2, net = res
        fp.write(json.dumps({"job": job.jid, "L": job.L, "p": job.p, "q": job.q, "t": int(t),
                             "s1": int(s1), "s2": int(s2), "n_sites": job.L * job.L, "w2": float(w2),
                             "net_flips": int(net), "since_arrival_s": clock() - job.arrival}) + "\n")
    return log


def summary(jobs, wall_s: float) -> dict:
    lat = sorted(j.latency for j in jobs)

    def pct(x):
        if not lat:
            return None
        i = min(len(lat) - 1, max(0, int(math.ceil(x / 100.0 * len(lat))) - 1))
        return lat[i]

    attempts = sum(j.attempts for j in jobs)
    return {"jobs": len(jobs), "p50_latency_s": pct(50), "p99_latency_s": pct(99),
            "attempts": attempts, "wall_s": wall_s, "attempts_per_ns": attempts / (wall_s * 1e9)}


class GpuBatch:
    """Adapter from the engine's batch interface to the C ABI batch."""

    def __init__(self, stream=None):
        from . import _address, _lib
        self._lib = _lib
        self._keep = stream
        self.h = _lib.oct_batch_create([], _address(stream, "cuda_stream"))

    def add(self, job: Job) -> int:
        r = self._lib.oct_replica()
        r.L, r.p, r.q, r.seed = job.L, job.p, job.q, job.seed
        r.Bx, r.By = job.shape
        return self._lib.oct_batch_add(self.h, r)

    def remove(self, slot: int) -> None:
        self._lib.oct_batch_remove(self.h, slot)

    def run(self, n: int) -> None:
        self._lib.oct_batch_run(self.h, n)

    def measure(self, slot: int):
        m = self._lib.oct_batch_measure_slot(self.h, slot)
        return (m.t, m.s1, m.s2, m.w2, m.net_flips)

    @staticmethod
    def _tuple(m):
        return (m.t, m.s1, m.s2, m.w2, m.net_flips)

    def measure_async(self, slot: int) -> int:
        return self._lib.oct_batch_measure_async(self.h, slot)

    def mark(self) -> int:
        return self._lib.oct_batch_mark(self.h)

    def mark_done(self, mark: int) -> bool:
        return self._lib.oct_batch_mark_done(self.h, mark)

    def wait_mark(self, mark: int) -> None:
        self._lib.oct_batch_mark_wait(self.h, mark)

    def poll(self, ticket: int):
        m = self._lib.oct_batch_poll(self.h, ticket)
        return None if m is None else self._tuple(m)

    def wait(self, ticket: int):
        return self._tuple(self._lib.oct_batch_wait(self.h, ticket))

    def close(self) -> None:
        if self.h:
            self._lib.oct_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
