"""Benchmark: octahedron-model DTrDT, site-update attempts per ns on GB300.

One step = one MCS (L^2 update attempts: four device steps of DTr plus
single-hit DT) over the whole lattice, resident in HBM.  Default workload:
L = 2^17 (1.7e10 sites, 4 GiB packed), KPZ with p = 0.95, q = 0.05, flat
start, seed 1 (+ rank), 1024 x 16-site sub-tiles, 4 x 4-site thread cells
(the DTrDB, DTrDTr and coarse-cell legs: 256 x 64-site sub-tiles).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica on its own GPU (the
method has no exchange between replicas); the value is the total attempts of
all ranks over the slowest rank's time.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "site-update attempts/ns at L=2^17 (plain vs batched) at bit-exact oracle match"
UNIT = "attempts/ns"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--L", type=int, default=2**17)
    ap.add_argument("--p", type=float, default=0.95)
    ap.add_argument("--q", type=float, default=0.05)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--Bx", type=int, default=1024)
    ap.add_argument("--By", type=int, default=16)
    ap.add_argument("--side-Bx", type=int, default=256, help="sub-tile of the DTrDB, DTrDTr and coarse-cell legs")
    ap.add_argument("--side-By", type=int, default=64)
    ap.add_argument("--e2e-steps", type=int, default=48)
    ap.add_argument("--e2e-lattices", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-cores", type=int, default=0, help="host cores for --impl reference (0: all)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch-replicas", type=int, default=2048)
    ap.add_argument("--batch-steps", type=int, default=100)
    ap.add_argument("--loop-steps", type=int, default=3)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=256)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-policy", default="large", help="autotune.batch_shape policy of the serving leg")
    ap.add_argument("--serve-inflight", type=int, default=4,
                    help="ticks the serving loop keeps enqueued ahead of the device per batch (0: no limit)")
    ap.add_argument("--serve-batches", type=int, default=1,
                    help="batches (streams) the serving loop spreads its jobs over")
    ap.add_argument("--db-steps", type=int, default=30)
    ap.add_argument("--cell-steps", type=int, default=2, help="timed MCS per coarse thread-cell shape")
    ap.add_argument("--ac-reps", type=int, default=5)
    ap.add_argument("--tune-mcs", type=int, default=1)
    ap.add_argument("--strips", action="store_true",
                    help="with N > 1 ranks: one lattice split into N row strips (strong scaling) "
                         "instead of N independent replicas")
    return ap.parse_args()


def workload(a):
    return {
        "workload": (f"octahedron model RS under DTrDT, L={a.L} ({a.L * a.L:.3g} sites, "
                     f"{a.L * a.L // 4 / 2**30:.3g} GiB packed), p={a.p} q={a.q}, flat start, "
                     f"{a.Bx}x{a.By}-site sub-tiles, 4x4-site thread cells, seed {a.seed}+rank"),
        "L": a.L, "p": a.p, "q": a.q, "Bx": a.Bx, "By": a.By, "cx": 4, "cy": 4,
        "form": "plain",
        "l2": "lattice larger than L2 (no flush needed)",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.device}",
                                       f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                v = [x.strip() for x in line.split(",")]
                if len(v) >= 9 and v[1].replace(".", "").isdigit():
                    rows.append(v)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(float(r[2]) for r in rows),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def philox_blocks_per_lane(scheme: str, cx: int, cy: int, random: bool) -> float:
    """Philox-4x32-10 blocks one lane of the plain device-step kernels
    evaluates per device step, apart from the tail stream (a lane holds 32 x 16
    sites, i.e. 512 attempts per device step): the MCS draw, the set draws
    (one block per 64 collective steps), the DTrDTr block origins (one block
    per 16 steps), the site words (DT: one block per 2 steps when two steps
    share a site field, else per step; DB: per step) and, with acceptance
    draws, the four level words (DT: one block per cx/4 steps, since a
    group of 32/cx cells per band uses 4*32/cx of a word's 32 bits per step;
    DB and DTrDTr: one block per step)."""
    steps = cx * cy
    bpt = (cx // 2).bit_length() - 1 + (cy // 2).bit_length() - 1
    spw = 2 if 2 * bpt <= cx else 1
    blocks = 1.0  # MCS draw
    if scheme == "DB":
        blocks += steps
    else:
        blocks += -(-steps // 64) + steps / spw
        if scheme == "DTR":
            blocks += -(-steps // 16)
    if random:
        blocks += steps / (cx // 4 if scheme == "DT" else 1)
    return blocks


def alu_accounting(scheme, cx, cy, random, attempts, tail_blocks, draws, tcs_per_subtile):
    """Integer operations per attempt, two ways.  Both charge 0.5 operations per
    random bit (Philox-4x32-10: ten rounds of about six operations per 128
    bits) plus 4 operations per attempt (the pattern test and the flip,
    amortised over a 32-site word):
      * generated: the bits the kernel actually generates (its Philox blocks
        per lane and device step, plus the tail-stream blocks it counted);
      * survey: the bits the method consumes as fixed before the first
        measurement (site offset + set draw + 32 bits per acceptance draw)."""
    gen_bits = 128.0 * philox_blocks_per_lane(scheme, cx, cy, random) / 512.0 + 128.0 * tail_blocks / attempts
    site_bits = (cx * cy).bit_length() - 1 if scheme == "DB" else (cx // 2 * cy // 2).bit_length() - 1
    shared = {"DB": 0.0, "DT": 2.0, "DTR": 6.0}[scheme]  # set (and DTrDTr origin) bits per collective step
    survey_bits = site_bits + shared / tcs_per_subtile + 32.0 * draws / attempts
    return {"generated": {"bits_per_attempt": gen_bits, "ops_per_attempt": 0.5 * gen_bits + 4.0},
            "survey": {"bits_per_attempt": survey_bits, "ops_per_attempt": 0.5 * survey_bits + 4.0}}


def step_traffic(src_hash: str, Bx: int, By: int, L: int):
    """DRAM bytes per device-step launch at this sub-tile shape and L from a
    committed ncu summary, if it was taken on the current kernel sources (else
    None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "dtrdt_step_traffic.json")) as f:
            d = json.load(f)
    except OSError:
        return None
    if d.get("kernel_sources_sha256") != src_hash:
        return None
    cap = d.get("captures", {}).get(f"{Bx}x{By}")
    if not cap:
        return None
    # traffic grows with the sites a launch updates
    return cap["dram_bytes_per_launch"] * (L / cap["captured_L"]) ** 2


STEP_SOURCES = ("dtrdt.cu", "subtile.cuh", "tiles.cuh", "philox.cuh")


def src_hash():
    """sha256 of the step kernel's source files with comments and blank lines
    removed (a comment edit does not invalidate a capture)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1705_01022_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(name.encode() + b"\0" + code.encode() + b"\0")
    return h.hexdigest()


def cpu_baseline_window(oracle, a, state_getter, t, target_s, scheme=0, seed=None, name="DTrDT", shape=None):
    """Times the oracle replaying MCS t on windows of the lattice (read from the
    running simulation), growing the window until about target_s of CPU work.
    shape: the sub-tile (Bx, By) of the run (default: the bench's)."""
    Bx, By = shape or (a.Bx, a.By)
    prm = oracle.Params(L=a.L, p=a.p, q=a.q, seed=a.seed if seed is None else seed, Bx=Bx, By=By,
                        scheme=scheme)
    tw, th = 2 * Bx, 2 * By
    ox, oy, _ = oracle.mcs_draw(prm, t)
    nx, ny, spent, attempts = 2, 2, 0.0, 0
    while True:
        nx = min(nx, a.L // tw)
        ny = min(ny, a.L // th)
        W, H = min(nx * tw + 1, a.L), min(ny * th + 1, a.L)
        Xw, Yw = state_getter(ox, oy, W, H)
        t0 = time.perf_counter()
        oracle.dtrdt_mcs_window(Xw, Yw, prm, t, ox, oy)
        dt = time.perf_counter() - t0
        spent, attempts = dt, nx * ny * tw * th
        if dt >= target_s * 0.5 or (nx * tw >= a.L and ny * th >= a.L):
            break
        grow = max(1.5, min(8.0, target_s / max(dt, 1e-3)))
        if nx <= ny:
            nx = int(nx * grow) + 1
        else:
            ny = int(ny * grow) + 1
    return {"value": attempts / (spent * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"oracle {name} replay of MCS {t} on a {nx}x{ny} device-tile window "
                       f"({attempts} attempts, {spent:.1f} s) of the GPU lattice state"),
            "_window": (prm, t, ox, oy, W, H, attempts)}


def _replay_task(task):
    """Host-core worker: replays MCS t of the oracle's schedule on a private
    copy of a window stored in a file; returns (attempts, replay seconds)."""
    import numpy as np

    import oracle
    path, H, W, prm, t, ox, oy, attempts = task
    view = np.memmap(path, dtype=np.uint8, mode="r", shape=(2, H, W))
    Xw, Yw = np.array(view[0]), np.array(view[1])
    del view
    t0 = time.perf_counter()
    oracle.dtrdt_mcs_window(Xw, Yw, prm, t, ox, oy)
    return attempts, time.perf_counter() - t0


def _warm_task(_):
    import oracle
    oracle.lib()
    return os.getpid()


class HostCores:
    """A process pool over the host cores (started with spawn, so it is safe
    after CUDA is up) in which every core replays its own copy of a window."""

    def __init__(self, n=None):
        import multiprocessing as mp
        self.n = n or len(os.sched_getaffinity(0))
        self.pool = mp.get_context("spawn").Pool(self.n)
        self.pool.map(_warm_task, range(self.n), chunksize=1)
        shm = "/dev/shm"
        self.dir = shm if os.path.isdir(shm) and os.access(shm, os.W_OK) else tempfile.gettempdir()

    def replay(self, Xw, Yw, prm, t, ox, oy, attempts):
        """All cores at once, one window copy each: (total attempts, wall s, per-core s)."""
        import numpy as np
        H, W = Xw.shape
        fd, path = tempfile.mkstemp(dir=self.dir, suffix=".win")
        os.close(fd)
        try:
            mm = np.memmap(path, dtype=np.uint8, mode="w+", shape=(2, H, W))
            mm[0], mm[1] = Xw, Yw
            mm.flush()
            del mm
            t0 = time.perf_counter()
            res = self.pool.map(_replay_task, [(path, H, W, prm, t, ox, oy, attempts)] * self.n, chunksize=1)
            wall = time.perf_counter() - t0
        finally:
            os.unlink(path)
        return sum(r[0] for r in res), wall, [r[1] for r in res]

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_all_cores(oracle, single, state_getter, name="DTrDT"):
    """The window of the single-core run, replayed by every host core at once
    (each on its own copy); the value is all attempts over the wall time,
    which includes the workers' copy of the window."""
    prm, t, ox, oy, W, H, attempts = single["_window"]
    Xw, Yw = state_getter(ox, oy, W, H)
    cores = HostCores()
    try:
        total, wall, per = cores.replay(Xw, Yw, prm, t, ox, oy, attempts)
    finally:
        cores.close()
    return {"value": total / (wall * 1e9), "unit": UNIT, "cores": cores.n, "kind": "oracle",
            "sample": (f"oracle {name} replay of MCS {t}: {cores.n} processes, each on its own copy of the "
                       f"window of the single-core sample ({attempts} attempts each, {wall:.1f} s wall, "
                       f"replays {min(per):.1f}-{max(per):.1f} s)"),
            "single_core": {k: v for k, v in single.items() if not k.startswith("_")}}


def cpu_sequential_rs(oracle, L=4096, p=1.0, q=0.0, seed=1, target_s=3.0):
    """O1 (sequential RS, one attempt at a time) on one core at L=4096, the
    paper's CPU comparison size (Sec. 4.3)."""
    X, Y = oracle.flat(L)
    n, spent = 0, 0.0
    while spent < target_s:
        t0 = time.perf_counter()
        oracle.seq_rs(X, Y, p, q, seed, n, 1)
        spent += time.perf_counter() - t0
        n += 1
    return {"value": n * L * L / (spent * 1e9), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle sequential RS (O1), L={L}, p={p}, q={q}, {n} MCS from the flat start, {spent:.1f} s"}


BATCH_PQ = [(1.0, 0.0), (0.95, 0.05), (0.5, 0.5)]


def batch_replicas(n, _lib, master=1):
    """Replica r: L drawn uniformly from {64, 128, ..., 4096} (numpy PCG64 seeded
    by the master seed), (p, q) cycled over the three pairs by index, key
    derived from the master seed with oct_replica_seed."""
    import numpy as np
    Ls = (np.random.default_rng(master).integers(1, 65, size=n) * 64).tolist()
    return [(int(Ls[r]), *BATCH_PQ[r % 3], _lib.oct_replica_seed(master, r)) for r in range(n)]


def batched_leg(a, g, _lib, torch, stream, peak_tops):
    """Many independent replicas of uneven L in one launch per device step and
    mode (graph replay), against a loop of plain per-replica launches."""
    from paper_1705_01022_gb300 import autotune
    reps = batch_replicas(a.batch_replicas, _lib)
    sites = sum(r[0] * r[0] for r in reps)
    # block tiles by the autotuner's batch policy (timed on this replica set)
    tuned = autotune.tune_batch(reps, mcs=4, stream=stream) if a.tune_mcs > 0 else None
    policy = tuned["policy"] if tuned else "default"
    shapes = [autotune.batch_shape(r[0], policy) for r in reps]
    reps = [r + sh for r, sh in zip(reps, shapes)]
    out = {"workload": (f"{len(reps)} replicas, L uniform in {{64,...,4096}} (multiples of 64), "
                        f"(p,q) cycled over {BATCH_PQ}, flat start, keys from master seed 1; "
                        f"sub-tiles by the autotuner's policy '{policy}'; 4x4 thread cells"),
           "replicas": len(reps), "sites": sites,
           "autotune": ({"policy": policy, "table": [[row["policy"], round(row["attempts_per_ns"], 1)]
                                                     for row in tuned["table"]]} if tuned else None)}
    with g.Batch(reps, stream=stream) as b:
        b.run(5)
        b.sync()
        t0 = b.stats()[3]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        b.run(a.batch_steps)
        end.record(stream)
        torch.cuda.synchronize()
        ms = start.elapsed_time(end)
        draws = b.stats()[3] - t0
        out.update({"value": sites * a.batch_steps / (ms * 1e6), "unit": UNIT,
                    "mcs": a.batch_steps, "ms_per_mcs": ms / a.batch_steps})
        # per-launch kernel time, launch by launch
        _lib.oct_batch_set_timing(b.h, True)
        b.run(5)
        kms, klaunch = _lib.oct_batch_get_timing(b.h)
        _lib.oct_batch_set_timing(b.h, False)
        f_draw = draws / (sites * a.batch_steps)
        # The batched kernel keeps no tail-block count: ties are 1/16 of the draws in
        # expectation and a block holds four tail words, so about draws/64 blocks.
        acct = alu_accounting("DT", 4, 4, True, 1.0, f_draw / 64.0, f_draw, 256)
        ops = acct["generated"]["ops_per_attempt"]
        achieved = ops * sites / 4 / (kms / klaunch * 1e-3) / 1e12
        survey = acct["survey"]["ops_per_attempt"] * sites / 4 / (kms / klaunch * 1e-3) / 1e12
        out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                           "frac": achieved / peak_tops, "kernel": "batch_step_kernel",
                           "device_step_ms": kms / klaunch, "draw_fraction": f_draw, "ops_per_attempt": ops,
                           "accounting": "generated bits; tail blocks estimated as draws/64",
                           "survey_accounting": {"ops_per_attempt": acct["survey"]["ops_per_attempt"],
                                                 "achieved": survey, "frac": survey / peak_tops}}
    # the same replicas, one plain handle each, launched one after another
    sims = [g.Simulation(L, p, q, seed, Bx=Bx, By=By, stream=stream) for (L, p, q, seed, Bx, By) in reps]
    for s_ in sims:
        s_.run(1)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(a.loop_steps):
        for s_ in sims:
            s_.run(1)
    end.record(stream)
    torch.cuda.synchronize()
    ms_loop = start.elapsed_time(end)
    for s_ in sims:
        s_.close()
    out["plain_loop"] = {"value": sites * a.loop_steps / (ms_loop * 1e6), "unit": UNIT,
                         "mcs": a.loop_steps,
                         "how": "one plain handle per replica, oct_run_mcs(1) per replica in turn, one stream"}
    out["batched_over_plain_loop"] = out["value"] / out["plain_loop"]["value"]
    out["gpu_launches_per_mcs"] = 9
    return out


def serving_leg(a, g, _lib, torch, stream, capacity):
    """Poisson streams of simulation jobs at offered loads of 0.5, 0.8 and 1.0
    times the batched capacity, served by continuous batching."""
    from paper_1705_01022_gb300 import serve
    work = serve.expected_work()
    out = {"workload": ("Poisson job stream: L log-uniform in [128, 16384] (multiples of 128), t_max "
                        "log-uniform in [10, 10^4] MCS, (p,q) uniform over (1,0), (0.8,0.2), (0.5,0.5), "
                        "W^2 streamed at 8 log-spaced times per job, HBM budget 64 GiB"),
           "shape_policy": a.serve_policy, "max_inflight_ticks": a.serve_inflight, "batches": a.serve_batches,
           "capacity_attempts_per_ns": capacity, "expected_attempts_per_job": work, "loads": []}
    # One job list (Poisson gaps of mean 1, keys from master seed 1).  The offered
    # load rho is the work the list actually holds per second of its arrival
    # span, over the capacity: arrival times are scaled so that the list's own
    # work arrives at rho x capacity (its work is heavy-tailed, so the expected
    # work per job would misstate the load of a finite list).
    base = serve.poisson_jobs(a.serve_jobs, 1.0, master_seed=1, seed_fn=_lib.oct_replica_seed)
    realized = sum(j.attempts for j in base)
    span = max(j.arrival for j in base)
    out.update({"jobs": len(base), "realized_attempts": realized,
                "realized_over_expected": realized / (len(base) * work),
                "offered_load_basis": "the job list's own work per second of arrival span / capacity"})
    for rho in (0.5, 0.8, 1.0):
        scale = realized / (rho * capacity * 1e9) / span
        jobs = [serve.Job(j.jid, j.L, j.p, j.q, j.seed, j.t_max, arrival=j.arrival * scale,
                          measure_at=list(j.measure_at)) for j in base]
        eng = serve.ServingEngine(64 << 30, stream=stream, max_chunk=64, shape_policy=a.serve_policy,
                                  max_inflight=a.serve_inflight, n_batches=a.serve_batches)
        t0 = time.perf_counter()
        done = eng.run(jobs)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        res = serve.summary(done, wall)
        res.update({"offered_load": rho, "rate_jobs_per_s": (len(base) - 1) / (span * scale), "ticks": eng.ticks,
                    "arrival_span_s": span * scale, "fraction_of_capacity": res["attempts_per_ns"] / capacity})
        out["loads"].append(res)
        eng.close()
    return out


def run_reference(a, rank, world):
    """The oracle as it stands, on the host cores, same metric and workload:
    each step, every core replays one MCS on its own copy of a bounded window
    of the lattice (flat start; the window follows the MCS origin)."""
    if rank != 0:
        return None
    import numpy as np

    import oracle
    oracle.build()
    prm = oracle.Params(L=a.L, p=a.p, q=a.q, seed=a.seed, Bx=a.Bx, By=a.By)
    tw, th = 2 * a.Bx, 2 * a.By
    nx, ny = max(1, min(a.L // tw, 8)), max(1, min(a.L // th, 4))
    W, H = min(nx * tw + 1, a.L), min(ny * th + 1, a.L)
    per_window = nx * ny * tw * th
    cores = HostCores(a.ref_cores or None)
    times, total = [], 0
    try:
        for step in range(a.warmup + a.steps):
            ox, oy, _ = oracle.mcs_draw(prm, step)
            xs = (ox + np.arange(W)) % a.L
            ys = (oy + np.arange(H)) % a.L
            flat = ((xs[None, :] + ys[:, None]) & 1).astype(np.uint8)
            n_att, wall, _ = cores.replay(flat, flat, prm, step, ox, oy, per_window)
            if step >= a.warmup:
                times.append(wall)
                total += n_att
    finally:
        cores.close()
    secs = sum(times)
    value = total / (secs * 1e9)
    sample = (f"oracle DTrDT replay of one MCS per step on {cores.n} host cores at once, each on its own copy "
              f"of a {nx}x{ny} device-tile window ({per_window} attempts per core and step) of the L={a.L} lattice")
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * secs / max(1, len(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": workload(a),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores.n, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def replica_seed(seed: int, rank: int) -> int:
    """Each rank runs an independent replica: its key is the base seed plus the rank."""
    return seed + rank


def combine_ranks(ms_local: float, attempts_local: int, dist=None, device="cpu"):
    """Slowest rank's time and total attempts over all ranks (weak scaling)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_local, attempts_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    n = torch.tensor([attempts_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def strips_main(a, rank, world, local, dist, torch, g, _lib):
    """Strong scaling: one L x L lattice split into `world` row strips, one per
    GPU, halo rows exchanged by NCCL between device steps (strips.py).  Prints
    one JSON line on rank 0."""
    from paper_1705_01022_gb300 import strips
    lay = strips.StripLayout(a.L, a.By, world, rank)
    eng = strips.GpuStripEngine(lay, a.p, a.q, a.seed, a.Bx)
    run = strips.StripRunner(lay, eng, a.seed, dist)
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()

    run.run(a.warmup)
    barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        run.run(a.steps)
        end.record(stream)
        barrier()
    ms = start.elapsed_time(end)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    w = run.measure()
    if rank == 0:
        cfg = workload(a)
        cfg.update({"form": "strips", "parallelism": f"strips{world}", "strip_rows": lay.H, "held_rows": lay.held})
        print(json.dumps({
            "metric": METRIC, "value": a.L * a.L * a.steps / (ms_max * 1e6), "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": cfg,
            "clocks": clk.summary(), "roofline": None, "cpu_baseline": None, "e2e": None,
            "gpu_launches": 4 * a.steps * world,
            "w2": {"t": w.t, "w2": w.w2, "s1": w.s1, "hmax": w.hmax, "how": "exact, combined from the strips"},
            "note": "one lattice over all ranks; halo rows by NCCL point-to-point between device steps"}),
              flush=True)
    eng.close()
    dist.destroy_process_group()


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        out = run_reference(a, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    import torch

    import paper_1705_01022_gb300 as g
    from paper_1705_01022_gb300 import _lib

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    g.build()
    if a.strips and world > 1:
        return strips_main(a, rank, world, local, dist, torch, g, _lib)
    # a dedicated stream: torch events and the library's kernels share it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    L = a.L
    lattice = torch.empty(L * L // 4, dtype=torch.uint8, device="cuda")
    seed = replica_seed(a.seed, rank)
    # ---- block-tile autotuner: every valid sub-tile shape at this L, its choice recorded ----
    tuning = None
    if rank == 0 and a.tune_mcs > 0:
        from paper_1705_01022_gb300 import autotune
        rec = autotune.tune(L, a.p, a.q, seed=seed, mcs=a.tune_mcs, stream=stream, lattice=lattice)
        tuning = {"choice": [rec["Bx"], rec["By"]], "cell": [rec["cx"], rec["cy"]], "mode": rec["mode"],
                  "device": rec["device"], "mcs_per_shape": rec["mcs"],
                  "table": [[r["Bx"], r["By"], round(r["attempts_per_ns"], 1)] for r in rec["table"]],
                  "bench_shape_is_choice": [rec["Bx"], rec["By"]] == [a.Bx, a.By]}
    sim = g.Simulation(L, a.p, a.q, seed, Bx=a.Bx, By=a.By, stream=stream, lattice=lattice)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    sim.run(a.warmup)
    barrier()
    stats0 = _lib.oct_get_stats(sim.h)
    _lib.oct_set_timing(sim.h, True)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        sim.run(a.steps)
        end.record(stream)
        barrier()
    ms = start.elapsed_time(end)
    step_ms, launches, _ = _lib.oct_get_timing(sim.h)
    _lib.oct_set_timing(sim.h, False)
    stats1 = _lib.oct_get_stats(sim.h)
    attempts = L * L * a.steps
    ms_max, total_attempts = combine_ranks(ms, attempts, dist, device="cuda")
    value = total_attempts / (ms_max * 1e6)

    # ---- roofline of the device-step kernel (integer-ALU bound) ----
    launch_ms = step_ms / max(1, launches)
    att_per_launch = L * L / 4
    tcs_per_subtile = (a.Bx // 4) * (a.By // 4)
    f_draw = (stats1.draws - stats0.draws) / attempts
    any_random = 0.0 < a.p < 1.0 or 0.0 < a.q < 1.0
    acct = alu_accounting("DT", 4, 4, any_random, attempts, stats1.tail_blocks - stats0.tail_blocks,
                          stats1.draws - stats0.draws, tcs_per_subtile)
    ops_per_attempt = acct["generated"]["ops_per_attempt"]
    lop3, probe_mhz, sms = _lib.oct_probe_int_rate(0)
    imad, _, _ = _lib.oct_probe_int_rate(1)
    pk = peaks()
    max_mhz = float(pk.get("sm_max_mhz", 2070.0))
    peak_tops = sms * lop3 * max_mhz * 1e6 / 1e12
    achieved_tops = ops_per_attempt * att_per_launch / (launch_ms * 1e-3) / 1e12
    survey_tops = acct["survey"]["ops_per_attempt"] * att_per_launch / (launch_ms * 1e-3) / 1e12
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    hbm_gbs = 2 * (L * L / 16) / (launch_ms * 1e-3) / 1e9  # quarter lattice read + written
    roofline = {
        "bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s",
        "frac": achieved_tops / peak_tops, "traffic": step_traffic(src_hash(), a.Bx, a.By, L),
        "traffic_vs_algorithmic": (lambda tr: tr / (2 * L * L / 16) if tr else None)(
            step_traffic(src_hash(), a.Bx, a.By, L)),
        "kernel": "dtrdt_step_kernel", "launch_ms": launch_ms, "launches": launches,
        "ops_per_attempt": ops_per_attempt, "draw_fraction": f_draw,
        "accounting": "generated: 0.5 op per random bit the kernel generates + 4 ops per attempt",
        "bits_per_attempt": acct["generated"]["bits_per_attempt"],
        "survey_accounting": {"ops_per_attempt": acct["survey"]["ops_per_attempt"],
                              "bits_per_attempt": acct["survey"]["bits_per_attempt"],
                              "achieved": survey_tops, "frac": survey_tops / peak_tops,
                              "note": "bits the method consumes (32 per acceptance draw), not those generated"},
        "peak_basis": (f"{sms} SMs x {lop3:.1f} LOP3/clk/SM (probe; IMAD {imad:.1f}) x "
                       f"{max_mhz:.0f} MHz max SM clock"),
        "hbm": {"achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_gbs / hbm_peak},
    }

    # ---- end to end through the C ABI with host buffers ----
    # (right after the timed region: after the other legs, the copies from
    # page-locked memory stalled for 0.1-0.2 s about every 0.3 s)
    # Each step copies one lattice in from page-locked host memory, runs one
    # MCS, measures W^2 and copies the lattice back out.  `--e2e-lattices`
    # independent lattices (the benchmark's own and replicas with seeds
    # seed + 1000 k, each on its own stream) take the steps in turn, driven
    # from one host thread with the asynchronous calls, so that one lattice's
    # copies overlap another's kernels and copies in the other direction.
    e2e = None
    if not a.no_e2e and a.e2e_steps > 0:
        words = L * L // 16
        # page-locked host memory: at most a quarter of the host's RAM over all ranks
        ram = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
        nl = max(1, min(a.e2e_lattices, int(0.25 * ram) // (world * 4 * words)))
        e2e_sims = [sim] + [g.Simulation(L, a.p, a.q, seed + 1000 * k, Bx=a.Bx, By=a.By)
                            for k in range(1, nl)]
        hosts = [torch.empty(words * 4, dtype=torch.uint8, pin_memory=True) for _ in range(nl)]
        _lib.oct_get_planes(sim.h, hosts[0].data_ptr(), words)
        for hb in hosts[1:]:
            hb.copy_(hosts[0])
        tk = [sim.t] * nl
        pending = [False] * nl

        marks = []  # host time (ms from the timed start) after each wait and each copy in, per step

        def e2e_step(i, t0=None):
            k = i % nl
            h = e2e_sims[k].h
            if pending[k]:
                _lib.oct_w2_wait(h)
            tw_ = time.perf_counter()
            _lib.oct_set_planes(h, hosts[k].data_ptr(), words, tk[k])
            ts_ = time.perf_counter()
            _lib.oct_run_mcs(h, 1)
            _lib.oct_measure_w2_async(h)
            _lib.oct_get_planes_async(h, hosts[k].data_ptr(), words)
            tk[k] += 1
            pending[k] = True
            if t0 is not None:
                marks.append([round((tw_ - t0) * 1e3, 1), round((ts_ - t0) * 1e3, 1)])

        def e2e_drain():
            for k in range(nl):
                if pending[k]:
                    _lib.oct_w2_wait(e2e_sims[k].h)
                    pending[k] = False

        for i in range(nl):  # one untimed step per lattice (first use of each host buffer)
            e2e_step(i)
        e2e_drain()
        barrier()
        t0 = time.perf_counter()
        for i in range(a.e2e_steps):
            e2e_step(i, t0)
        e2e_drain()
        barrier()
        e2e_s = time.perf_counter() - t0
        for extra in e2e_sims[1:]:
            extra.close()
        if dist is not None:
            t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        # one more step, phase by phase, for the breakdown
        ph = []
        hp = hosts[0].data_ptr()
        for fn in (lambda: _lib.oct_set_planes(sim.h, hp, words, sim.t), lambda: sim.run(1),
                   lambda: sim.measure(), lambda: _lib.oct_get_planes(sim.h, hp, words)):
            sim.sync()
            t1 = time.perf_counter()
            fn()
            sim.sync()
            ph.append(time.perf_counter() - t1)
        e2e = {"value": world * L * L * a.e2e_steps / (e2e_s * 1e9), "unit": UNIT,
               "h2d_bytes_per_step": L * L // 4, "d2h_bytes_per_step": L * L // 4 + 56,
               "steps": a.e2e_steps, "lattices_in_flight": nl, "host_marks_ms": marks,
               "copy_in_ms_median": statistics.median(b - w for w, b in marks) if marks else None,
               "stalled_copies_in": sum(1 for w, b in marks if marks and b - w > 2 * statistics.median(
                   b2 - w2 for w2, b2 in marks)),
               "breakdown_ms": {"h2d": ph[0] * 1e3, "mcs": ph[1] * 1e3, "measure_w2": ph[2] * 1e3,
                                "d2h": ph[3] * 1e3},
               "h2d_gbs": (L * L // 4) / ph[0] / 1e9, "d2h_gbs": (L * L // 4) / ph[3] / 1e9,
               "path": ("per step, lattice k = step mod lattices_in_flight: oct_set_planes(pinned host) + "
                        "oct_run_mcs(1) + oct_measure_w2_async + oct_get_planes_async(pinned host); "
                        "oct_w2_wait before the lattice's next step and at the end"),
               "breakdown_note": "one step of one lattice, phase by phase with a synchronisation between phases"}

    # ---- the DTrDB block layer on the same workload (the paper's Fig. 7 pair) ----
    dtrdb = dtrdtr = cells = None
    if rank == 0 and a.db_steps > 0:
        sim.close()

        def timed(p, q, scheme, n, oracle_scheme=None):
            # continues from the lattice as it stands (no_init), new time origin
            with g.Simulation(L, p, q, seed, Bx=a.side_Bx, By=a.side_By, stream=stream, lattice=lattice,
                              no_init=True, scheme=scheme) as h:
                h.run(2)
                torch.cuda.synchronize()
                st0 = _lib.oct_get_stats(h.h)
                _lib.oct_set_timing(h.h, True)
                st_, en_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                st_.record(stream)
                h.run(n)
                en_.record(stream)
                torch.cuda.synchronize()
                kms, kl, _ = _lib.oct_get_timing(h.h)
                st1 = _lib.oct_get_stats(h.h)
                step_ms = kms / max(1, kl)
                f_draw = (st1.draws - st0.draws) / (L * L * n)
                tails_[0] = (st1.tail_blocks - st0.tail_blocks) / (L * L * n)
                cpu_ = None
                if oracle_scheme is not None and not a.no_cpu and world == 1:
                    import oracle
                    oracle.build()
                    cpu_ = cpu_baseline_window(oracle, a, lambda x, y, W, H: h.window(x, y, W, H), h.t,
                                               a.cpu_seconds / 4, scheme=oracle_scheme, seed=seed,
                                               name={1: "DTrDB", 3: "DTrDTr"}[oracle_scheme],
                                               shape=(a.side_Bx, a.side_By))
                    cpu_.pop("_window")
            return L * L * n / (st_.elapsed_time(en_) * 1e6), step_ms, f_draw, cpu_

        tails_ = [0.0]  # tail-stream blocks per attempt of the last timed run

        def alu_roofline(step_ms, scheme, f_draw, tail_per_attempt):
            acc = alu_accounting(scheme, 4, 4, any_random, 1.0, tail_per_attempt, f_draw, tcs)
            ops = acc["generated"]["ops_per_attempt"]
            ach = ops * (L * L / 4) / (step_ms * 1e-3) / 1e12
            sv = acc["survey"]["ops_per_attempt"] * (L * L / 4) / (step_ms * 1e-3) / 1e12
            return {"bound": "alu", "achieved": ach, "peak": peak_tops, "unit": "Tops/s", "frac": ach / peak_tops,
                    "ops_per_attempt": ops, "bits_per_attempt": acc["generated"]["bits_per_attempt"],
                    "launch_ms": step_ms,
                    "survey_accounting": {"ops_per_attempt": acc["survey"]["ops_per_attempt"],
                                          "achieved": sv, "frac": sv / peak_tops}}

        tcs = (a.side_Bx // 4) * (a.side_By // 4)
        db_v, db_step, db_f, db_cpu = timed(a.p, a.q, _lib.OCT_SCHEME_DB, a.db_steps, oracle_scheme=1)
        db_tail = tails_[0]
        kdt_v, kdt_step, _, _ = timed(1.0, 0.0, _lib.OCT_SCHEME_DT, a.db_steps)
        kdb_v, kdb_step, _, _ = timed(1.0, 0.0, _lib.OCT_SCHEME_DB, a.db_steps)
        dtrdb = {"value": db_v, "unit": UNIT, "mcs": a.db_steps, "device_step_ms": db_step,
                 "sub_tile": [a.side_Bx, a.side_By],
                 "scheme": "DTrDB: single-hit dead border at block level, borders delayed (p, q > 0)",
                 "start": "the DTrDT state after the timed region and the end-to-end steps",
                 "relative_to_dtrdt": db_v / (value / world),
                 "roofline": dict(alu_roofline(db_step, "DB", db_f, db_tail), draw_fraction=db_f,
                                  kernel="dtrdt_step_kernel<1, 2>"),
                 "cpu_baseline": db_cpu,
                 "kpz": {"p": 1.0, "q": 0.0, "dtrdt": kdt_v, "dtrdb": kdb_v, "relative": kdb_v / kdt_v,
                         "device_step_ms": {"dtrdt": kdt_step, "dtrdb": kdb_step},
                         "note": "DB with one rate zero carries out all attempts of a step together"}}
        dtr_v, dtr_step, dtr_f, dtr_cpu = timed(a.p, a.q, _lib.OCT_SCHEME_DTR, a.db_steps, oracle_scheme=3)
        dtr_tail = tails_[0]
        dtrdtr = {"value": dtr_v, "unit": UNIT, "mcs": a.db_steps, "device_step_ms": dtr_step,
                  "sub_tile": [a.side_Bx, a.side_By],
                  "scheme": "DTrDTr: double tiling with a block-layer origin moved after every collective step",
                  "start": "the DTrDB state after its run", "relative_to_dtrdt": dtr_v / (value / world),
                  "roofline": dict(alu_roofline(dtr_step, "DTR", dtr_f, dtr_tail), draw_fraction=dtr_f,
                                   kernel="dtrdt_step_kernel<1, 3>"),
                  "cpu_baseline": dtr_cpu}
        # ---- DTrDT with the paper's coarser thread cells (TC=1,1 .. 3,2) on the same workload ----
        cells = {}
        for cx, cy in (((4, 4), (8, 8), (16, 8), (16, 16), (32, 16)) if a.cell_steps > 0 else ()):
            with g.Simulation(L, a.p, a.q, seed, Bx=a.side_Bx, By=a.side_By, cx=cx, cy=cy, stream=stream,
                              lattice=lattice,
                              no_init=True) as h:
                h.run(1)
                torch.cuda.synchronize()
                st0 = _lib.oct_get_stats(h.h)
                _lib.oct_set_timing(h.h, True)
                st_, en_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                st_.record(stream)
                h.run(a.cell_steps)
                en_.record(stream)
                torch.cuda.synchronize()
                kms, kl, _ = _lib.oct_get_timing(h.h)
                st1 = _lib.oct_get_stats(h.h)
                n_att = L * L * a.cell_steps
                acc_ = alu_accounting("DT", cx, cy, any_random, n_att, st1.tail_blocks - st0.tail_blocks,
                                      st1.draws - st0.draws, (a.side_Bx // cx) * (a.side_By // cy))
                step_ = kms / max(1, kl)
                ach = acc_["generated"]["ops_per_attempt"] * (L * L / 4) / (step_ * 1e-3) / 1e12
                cells[f"{cx}x{cy}"] = {
                    "value": n_att / (st_.elapsed_time(en_) * 1e6), "unit": UNIT, "device_step_ms": step_,
                    "paper_tc": f"TC={(cx // 4).bit_length() - 1},{(cy // 4).bit_length() - 1}",
                    "roofline": {"bound": "alu", "achieved": ach, "peak": peak_tops, "frac": ach / peak_tops,
                                 "ops_per_attempt": acc_["generated"]["ops_per_attempt"],
                                 "bits_per_attempt": acc_["generated"]["bits_per_attempt"]}}
        if cells:
            # the cell tuner's choice on these rates: the fastest cell whose W^2 (ensemble of small
            # lattices at this p, q) lies within 1 % of the coarsest cell's
            from paper_1705_01022_gb300 import autotune
            rates = {tuple(int(v) for v in k.split("x")): c["value"] for k, c in cells.items()}
            rec = autotune.tune_cell(L, a.p, a.q, a.side_Bx, a.side_By, max_shift=0.01, cells=list(rates),
                                     measure_fn=lambda c: rates[c], stream=stream)
            cells["sub_tile"] = [a.side_Bx, a.side_By]
            cells["tuner"] = {"max_shift": rec["max_shift"], "choice": [rec["cx"], rec["cy"]],
                              "reference": rec["reference"], "fidelity_ensemble": rec["stat"],
                              "table": [[r["cx"], r["cy"], round(r["attempts_per_ns"], 1),
                                         [round(x, 4) for x in r["w2_ratio"]]] for r in rec["table"]]}
        sim = g.Simulation(L, a.p, a.q, seed, Bx=a.Bx, By=a.By, stream=stream, lattice=lattice)
        sim.run(a.warmup + a.steps)

    # ---- exact roughness W^2 (Eq. (3)) on the live state ----
    w2_leg = None
    if rank == 0 and a.ac_reps > 0:
        m = sim.measure()
        st_, en_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st_.record(stream)
        for _ in range(a.ac_reps):
            m = sim.measure()
        en_.record(stream)
        torch.cuda.synchronize()
        w2_ms = st_.elapsed_time(en_) / a.ac_reps
        w2_bytes = L * L // 8 + 4 * L  # the X plane and one Y word per row, read once
        w2_gbs = w2_bytes / (w2_ms * 1e-3) / 1e9
        w2_cpu = None
        if not a.no_cpu and world == 1:
            import oracle
            oracle.build()
            Lc = 2048
            Xc, Yc = oracle.flat(Lc)
            oracle.dtrdt_run(Xc, Yc, oracle.Params(L=Lc, p=a.p, q=a.q, seed=seed, Bx=256, By=64), 0, 2)
            reps_c, t0c = 0, time.perf_counter()
            while reps_c < 3 or time.perf_counter() - t0c < 1.0:
                oracle.w2_sums(Xc, Yc)
                reps_c += 1
            sec_c = (time.perf_counter() - t0c) / reps_c
            w2_cpu = {"value": Lc * Lc / (sec_c * 1e9), "unit": "sites/ns", "cores": 1, "kind": "oracle",
                      "sample": f"oracle O3 (exact S1, S2) on an L={Lc} lattice after 2 MCS, {reps_c} calls"}
        w2_leg = {"t": m.t, "w2": m.w2, "ms_per_call": w2_ms, "sites_per_ns": L * L / (w2_ms * 1e6),
                  "calls": a.ac_reps, "cpu_baseline": w2_cpu,
                  "roofline": {"bound": "hbm", "achieved": w2_gbs, "peak": hbm_peak, "unit": "GB/s",
                               "frac": w2_gbs / hbm_peak, "algorithmic_bytes": w2_bytes},
                  "note": "per oct_measure_w2 call: flip-counter sum, row pass, final pass, read-back and "
                          "synchronisation"}

    # ---- two-time autocorrelations C_h, C_s (Sec. 2) on the live state ----
    two_time = None
    if rank == 0 and a.ac_reps > 0:
        sim.snapshot()
        sim.run(1)
        ac = sim.measure_ac()
        st_, en_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st_.record(stream)
        for _ in range(a.ac_reps):
            ac = sim.measure_ac()
        en_.record(stream)
        torch.cuda.synchronize()
        ac_ms = st_.elapsed_time(en_) / a.ac_reps
        ac_bytes = L * L // 2  # both planes of both lattices, read once
        ac_gbs = ac_bytes / (ac_ms * 1e-3) / 1e9
        ac_cpu = None
        if not a.no_cpu and world == 1:
            import numpy as np
            import oracle
            oracle.build()
            Lc = 2048  # the oracle's lattices: flat start, 2 and 3 MCS of DTrDT
            prm_c = oracle.Params(L=Lc, p=a.p, q=a.q, seed=seed, Bx=256, By=64)
            Xs, Ys = oracle.flat(Lc)
            oracle.dtrdt_run(Xs, Ys, prm_c, 0, 2)
            Xt, Yt = Xs.copy(), Ys.copy()
            oracle.dtrdt_run(Xt, Yt, prm_c, 2, 1)
            reps_c, t0c = 0, time.perf_counter()
            while reps_c < 3 or time.perf_counter() - t0c < 1.0:
                oracle.two_time(Xt, Yt, Xs, Ys)
                reps_c += 1
            cpu_s = (time.perf_counter() - t0c) / reps_c
            ac_cpu = {"value": Lc * Lc / (cpu_s * 1e9), "unit": "sites/ns", "cores": 1, "kind": "oracle",
                      "sample": f"oracle two-time sums of two L={Lc} lattices, {reps_c} calls, {cpu_s * 1e3:.1f} ms each"}
        two_time = {"t": ac.t, "s": ac.s, "c_h": ac.c_h, "c_s": ac.c_s, "ms_per_call": ac_ms,
                    "sites_per_ns": L * L / (ac_ms * 1e6), "cpu_baseline": ac_cpu,
                    "calls": a.ac_reps,
                    "roofline": {"bound": "hbm", "achieved": ac_gbs, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": ac_gbs / hbm_peak, "algorithmic_bytes": ac_bytes},
                    "note": "per oct_measure_ac call: row pass, final pass and the 80-byte read-back"}

    # ---- batched replicas (uneven L) against a loop of plain launches ----
    batched = None
    if rank == 0 and not a.no_batch and a.batch_replicas > 0:
        batched = batched_leg(a, g, _lib, torch, stream, peak_tops)

    # ---- serving: continuous batching of a Poisson job stream ----
    serving = None
    if rank == 0 and not a.no_serve and a.serve_jobs > 0:
        cap = batched["value"] if batched else value
        serving = serving_leg(a, g, _lib, torch, stream, cap)

    # ---- CPU baseline: the oracle on a sample of the same state ----
    # (last: run right after the worker processes had exited, the first
    # end-to-end copies from page-locked memory were up to 7x slower)
    # One core first (sizes the window to about --cpu-seconds), then every
    # host core on its own copy of that window; O1 beside it at L=4096.
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu:
        import oracle
        oracle.build()

        def getter(x, y, W, H):
            return sim.window(x, y, W, H)

        single = cpu_baseline_window(oracle, a, getter, sim.t, a.cpu_seconds)
        cpu = cpu_baseline_all_cores(oracle, single, getter)
        cpu["sequential_rs_L4096"] = cpu_sequential_rs(oracle)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload(a), "clocks": clk.summary(), "roofline": roofline,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 5 * a.steps, "autotune": tuning, "dtrdb": dtrdb, "dtrdtr": dtrdtr, "cells": cells, "w2": w2_leg, "two_time": two_time, "batched": batched, "serving": serving,
            "probe": {"lop3_per_clk_per_sm": lop3, "imad_per_clk_per_sm": imad, "probe_mhz": probe_mhz},
        }
        print(json.dumps(out), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
