"""Autotuner for the block tile (the sub-tile of the device layer, Bx x By
sites) and the thread cell (cx x cy sites) of DTrDT.

The sub-tile shape is a parameter of the domain decomposition, not only of the
launch: it decides which sites are updated together and how the random
streams map onto sites (Sec. 3; the paper reports that the decomposition's
domain sizes shift the roughness prefactor, Sec. 4.2).  A tuned run is
therefore reproducible only with the same choice, so the tuner records it:
every decision is kept in a JSON cache keyed by GPU, L and acceptance mode,
together with the table it was taken from, and a later lookup returns the same
shape without measuring again.

For batched replicas (`tune_batch`) the shape is chosen per replica by a
policy (the library default, or the largest group count, wide or square), and
the policies are timed on the actual replica set: what a warp carries and how
the batched kernel packs it depend on the whole mix, not on one L.

Candidates are the shapes the step kernel accepts for this L: Bx a multiple of
32 and By a multiple of 16 (timed with 4 x 4-site thread cells), at most 32
groups of 32 x 16 sites, and L a multiple of 2Bx and 2By.  By default the
group counts in x and y are powers of two, which is also what a batched
replica needs.  Each candidate runs a warm-up MCS and then `mcs` timed MCS on
the library's own per-launch CUDA-event timing; the score is attempts per ns
of the device-step kernel.

The thread cell (`tune_cell`) is a choice between speed and fidelity, not
speed alone: finer cells run faster (more attempts per lane and step) but
lower the roughness prefactor below that of sequential RS (Sec. 4.2), while
coarse cells are indistinguishable from sequential runs (Sec. 5).  The tuner
therefore measures both on the GPU: the device-step rate of every supported
cell at the job's L and sub-tile, and each cell's W^2 on an ensemble of small
lattices at the job's p and q, relative to the coarsest cell (the stand-in for
RS, which has no parallel form).  It returns the fastest cell whose relative
W^2 lies within `max_shift` of 1 at every measured time, and records the whole
table like the sub-tile choice.
"""
from __future__ import annotations

import json
import os
import time
from dataclasses import dataclass, field

CELL = (4, 4)   # thread-cell shape (cx, cy) the sub-tile is timed with
# thread cells of the GPU's DTrDT block layer, finest first; the last is the
# coarsest (the fidelity reference of tune_cell)
CELLS = ((4, 4), (8, 4), (4, 8), (8, 8), (16, 4), (4, 16), (16, 8), (8, 16), (32, 4), (16, 16), (32, 8), (32, 16))
GROUP = (32, 16)  # sites held by one warp lane
MAX_GROUPS = 32


def mode_of(p: float, q: float) -> str:
    """'random' when an acceptance draw is needed (0 < p < 1 or 0 < q < 1), else 'deterministic'."""
    return "random" if (0.0 < p < 1.0) or (0.0 < q < 1.0) else "deterministic"


def candidates(L: int, pow2: bool = True) -> list[tuple[int, int]]:
    """Valid (Bx, By) for lattice size L, ordered by (Bx*By, Bx) descending."""
    out = []
    for gx in range(1, MAX_GROUPS + 1):
        for gy in range(1, MAX_GROUPS // gx + 1):
            if pow2 and (gx & (gx - 1) or gy & (gy - 1)):
                continue
            Bx, By = GROUP[0] * gx, GROUP[1] * gy
            if L % (2 * Bx) or L % (2 * By):
                continue
            out.append((Bx, By))
    out.sort(key=lambda s: (-s[0] * s[1], -s[0]))
    return out


def pick(table: list[dict]) -> dict:
    """Fastest entry; ties go to the larger sub-tile, then the wider one
    (the order of `candidates`), so the choice does not depend on dict order."""
    best = None
    for row in table:
        if best is None or row["attempts_per_ns"] > best["attempts_per_ns"]:
            best = row
    return best


def device_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name(torch.cuda.current_device())
    except Exception:  # noqa: BLE001 - torch is optional here
        pass
    return "cuda"


@dataclass
class TuneCache:
    """Recorded choices, one per (device, L, mode); stored as JSON at `path`
    (None: kept in memory only)."""
    path: str | None = None
    entries: dict = field(default_factory=dict)

    @staticmethod
    def key(device: str, L: int, mode: str) -> str:
        return f"{device}|L={L}|{mode}"

    @classmethod
    def load(cls, path: str | None) -> "TuneCache":
        c = cls(path)
        if path and os.path.exists(path):
            with open(path) as f:
                c.entries = json.load(f)
        return c

    def get(self, device: str, L: int, mode: str):
        return self.entries.get(self.key(device, L, mode))

    def put(self, record: dict) -> None:
        self.put_key(self.key(record["device"], record["L"], record["mode"]), record)

    def put_key(self, key: str, record: dict) -> None:
        self.entries[key] = record
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def measure(L: int, p: float, q: float, Bx: int, By: int, seed: int = 1, mcs: int = 2,
            stream=None, lattice=None, cx: int = 4, cy: int = 4) -> float:
    """Attempts per ns of the device-step kernel for one shape (flat start,
    one warm-up MCS, then `mcs` timed MCS)."""
    from . import Simulation, _lib
    with Simulation(L, p, q, seed, Bx=Bx, By=By, cx=cx, cy=cy, stream=stream, lattice=lattice) as sim:
        sim.run(1)
        sim.sync()
        _lib.oct_set_timing(sim.h, True)
        sim.run(mcs)
        sim.sync()
        ms, launches, _ = _lib.oct_get_timing(sim.h)
    per_launch_ms = ms / max(1, launches)
    return (L * L / 4.0) / (per_launch_ms * 1e6)


def tune(L: int, p: float, q: float, seed: int = 1, mcs: int = 2, shapes=None, stream=None,
         lattice=None, measure_fn=None) -> dict:
    """Measures every candidate shape and returns the record of the choice:
    {device, L, p, q, mode, Bx, By, cx, cy, attempts_per_ns, table, mcs, seed, when}."""
    shapes = list(shapes) if shapes is not None else candidates(L)
    if not shapes:
        raise ValueError(f"no sub-tile shape fits L={L}")
    fn = measure_fn or (lambda Bx, By: measure(L, p, q, Bx, By, seed, mcs, stream, lattice))
    table = [{"Bx": Bx, "By": By, "attempts_per_ns": float(fn(Bx, By))} for Bx, By in shapes]
    best = pick(table)
    return {"device": device_name() if measure_fn is None else "test", "L": L, "p": p, "q": q,
            "mode": mode_of(p, q), "Bx": best["Bx"], "By": best["By"], "cx": CELL[0], "cy": CELL[1],
            "attempts_per_ns": best["attempts_per_ns"], "table": table, "mcs": mcs, "seed": seed,
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


def choose(L: int, p: float, q: float, cache: TuneCache | None = None, **kw) -> dict:
    """The recorded choice for (GPU, L, mode), measuring once if there is none."""
    cache = cache if cache is not None else TuneCache()
    dev = device_name() if kw.get("measure_fn") is None else "test"
    rec = cache.get(dev, L, mode_of(p, q))
    if rec is None:
        rec = tune(L, p, q, **kw)
        cache.put(rec)
    return rec


def tuned_simulation(L: int, p: float, q: float, seed: int, cache: TuneCache | None = None,
                     stream=None, lattice=None, max_shift: float | None = None, **kw):
    """A Simulation on the tuned (recorded) sub-tile shape; the record is
    attached as `.tuning`.  With `max_shift`, the thread cell is tuned too
    (`choose_cell` on the tuned sub-tile) and its record attached as
    `.cell_tuning`; else the cell is 4 x 4 sites."""
    from . import Simulation
    cache = cache if cache is not None else TuneCache()
    rec = choose(L, p, q, cache=cache, stream=stream, **kw)
    cell, crec = CELL, None
    if max_shift is not None:
        crec = choose_cell(L, p, q, rec["Bx"], rec["By"], max_shift=max_shift, cache=cache, stream=stream,
                           mcs=kw.get("mcs", 1))
        cell = (crec["cx"], crec["cy"])
    sim = Simulation(L, p, q, seed, Bx=rec["Bx"], By=rec["By"], cx=cell[0], cy=cell[1], stream=stream,
                     lattice=lattice)
    sim.tuning = rec
    sim.cell_tuning = crec
    return sim


# ---------------------------------------------------------------------------
# thread cell: speed against fidelity
STAT_L = 256          # lattice size of the fidelity ensemble
STAT_SEEDS = 32       # realizations per cell
STAT_TIMES = (4, 16)  # MCS at which W^2 is compared
STAT_SHAPE = (64, 64)  # sub-tile of the fidelity ensemble


def ensemble_w2(p: float, q: float, cell, L: int = STAT_L, seeds: int = STAT_SEEDS, times=STAT_TIMES,
                seed0: int = 1, shape=STAT_SHAPE, stream=None) -> list[list[float]]:
    """W^2 at `times` for `seeds` realizations (seeds seed0 .. seed0+seeds-1)
    of DTrDT with thread cell `cell` from the flat start: a seeds x len(times)
    list."""
    from . import Simulation
    out = []
    for i in range(seeds):
        row, t = [], 0
        with Simulation(L, p, q, seed0 + i, Bx=shape[0], By=shape[1], cx=cell[0], cy=cell[1],
                        stream=stream) as sim:
            for tt in times:
                sim.run(tt - t)
                t = tt
                row.append(float(sim.measure().w2))
        out.append(row)
    return out


def relative_w2(cell_w2, ref_w2) -> list[tuple[float, float]]:
    """(mean W^2 of the cell / mean W^2 of the reference, standard error of
    the ratio) at each time, the two ensembles independent."""
    import statistics
    res = []
    for j in range(len(cell_w2[0])):
        a = [r[j] for r in cell_w2]
        b = [r[j] for r in ref_w2]
        ma, mb = statistics.fmean(a), statistics.fmean(b)
        va = statistics.variance(a) / len(a) if len(a) > 1 else 0.0
        vb = statistics.variance(b) / len(b) if len(b) > 1 else 0.0
        ratio = ma / mb
        res.append((ratio, abs(ratio) * (va / ma ** 2 + vb / mb ** 2) ** 0.5))
    return res


def pick_cell(table: list[dict], max_shift: float) -> dict:
    """The fastest row whose relative W^2 lies within max_shift of 1 at every
    time; the reference row (shift 0 by definition) always qualifies."""
    ok = [r for r in table if all(abs(x - 1.0) <= max_shift for x in r["w2_ratio"])]
    return max(ok, key=lambda r: r["attempts_per_ns"])


def tune_cell(L: int, p: float, q: float, Bx: int, By: int, max_shift: float = 0.01, seed: int = 1,
              mcs: int = 1, cells=CELLS, stream=None, measure_fn=None, w2_fn=None) -> dict:
    """Measures every cell's device-step rate at (L, Bx, By) and its W^2
    relative to the coarsest cell on the fidelity ensemble, and returns the
    record of the choice: {device, L, p, q, Bx, By, cx, cy, attempts_per_ns,
    max_shift, reference, table, stat, when}."""
    cells = [tuple(c) for c in cells]
    ref = max(cells, key=lambda c: (c[0] * c[1], c[0]))
    fn = measure_fn or (lambda c: measure(L, p, q, Bx, By, seed, mcs, stream, cx=c[0], cy=c[1]))
    wfn = w2_fn or (lambda c: ensemble_w2(p, q, c, stream=stream))
    ref_w2 = wfn(ref)
    table = []
    for c in cells:
        rel = [(1.0, 0.0)] * len(ref_w2[0]) if c == ref else relative_w2(wfn(c), ref_w2)
        table.append({"cx": c[0], "cy": c[1], "attempts_per_ns": float(fn(c)),
                      "w2_ratio": [r for r, _ in rel], "w2_ratio_err": [e for _, e in rel]})
    best = pick_cell(table, max_shift)
    return {"device": device_name() if measure_fn is None else "test", "L": L, "p": p, "q": q,
            "Bx": Bx, "By": By, "cx": best["cx"], "cy": best["cy"], "attempts_per_ns": best["attempts_per_ns"],
            "max_shift": max_shift, "reference": list(ref), "table": table,
            "stat": {"L": STAT_L, "seeds": STAT_SEEDS, "times": list(STAT_TIMES), "shape": list(STAT_SHAPE)},
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


def cell_key(device: str, L: int, p: float, q: float, Bx: int, By: int, max_shift: float) -> str:
    return f"{device}|L={L}|p={p!r}|q={q!r}|{Bx}x{By}|cell|max_shift={max_shift!r}"


def choose_cell(L: int, p: float, q: float, Bx: int, By: int, max_shift: float = 0.01,
                cache: TuneCache | None = None, **kw) -> dict:
    """The recorded cell choice for (GPU, L, p, q, sub-tile, max_shift),
    measuring once if there is none."""
    cache = cache if cache is not None else TuneCache()
    dev = device_name() if kw.get("measure_fn") is None else "test"
    key = cell_key(dev, L, p, q, Bx, By, max_shift)
    rec = cache.entries.get(key)
    if rec is None:
        rec = tune_cell(L, p, q, Bx, By, max_shift=max_shift, **kw)
        cache.put_key(key, rec)
    return rec


# ---------------------------------------------------------------------------
# batched replicas
BATCH_POLICIES = ("default", "wide", "square", "tall", "large")
LARGE_MIN_SUBTILES = 1024  # sub-tiles per device step for which 'large' keeps the wide shape


def groups(shape: tuple[int, int]) -> int:
    return (shape[0] // GROUP[0]) * (shape[1] // GROUP[1])


def batch_shape(L: int, policy: str) -> tuple[int, int]:
    """Sub-tile of a replica of size L under a policy: 'default' is the batch
    library's own default (64 x 64 if L % 128 == 0, else 32 x 32); 'wide' and
    'square' take the most groups a valid shape allows, then the widest or the
    most nearly square one; 'tall' takes 'wide' where that fills a warp, else
    the one-group-wide shape with the most groups (its lanes exchange no
    columns); 'large' takes the wide shape where it still leaves
    at least LARGE_MIN_SUBTILES sub-tiles per device step (large lattices get
    full-warp sub-tiles, as in the plain kernel), else the default."""
    if policy == "default":
        return (64, 64) if L % 128 == 0 else (32, 32)
    if policy == "large":
        Bx, By = batch_shape(L, "wide")
        if (L // (2 * Bx)) * (L // (2 * By)) >= LARGE_MIN_SUBTILES:
            return (Bx, By)
        return batch_shape(L, "default")
    shapes = candidates(L)
    if not shapes:
        raise ValueError(f"no sub-tile shape fits L={L}")
    gmax = max(groups(sh) for sh in shapes)
    best = [sh for sh in shapes if groups(sh) == gmax]
    if policy == "wide":
        return max(best, key=lambda sh: sh[0])
    if policy == "square":
        return min(best, key=lambda sh: (abs(sh[0].bit_length() - sh[1].bit_length()), -sh[0]))
    if policy == "tall":
        if gmax == MAX_GROUPS:  # full warps: as 'wide'
            return max(best, key=lambda sh: sh[0])
        return max((sh for sh in shapes if sh[0] == GROUP[0]), key=groups)
    raise ValueError(f"unknown policy {policy!r}")


def batch_key(replicas) -> str:
    """Digest of the replica mix (L and acceptance mode of every replica)."""
    import hashlib
    items = sorted((int(r[0]), mode_of(float(r[1]), float(r[2]))) for r in replicas)
    return hashlib.sha256(repr(items).encode()).hexdigest()[:16]


def measure_batch(replicas, mcs: int = 4, stream=None) -> float:
    """Attempts per ns of mcs batched MCS as they run (the captured graphs,
    whose branches overlap on the device), after a warm-up run of the same
    length that captures them, for replicas (L, p, q, seed, Bx, By)."""
    from . import Batch
    sites = sum(int(r[0]) ** 2 for r in replicas)
    with Batch(replicas, stream=stream) as b:
        b.run(mcs)
        b.sync()
        t0 = time.perf_counter()
        b.run(mcs)
        b.sync()
        dt = time.perf_counter() - t0
    return sites * mcs / (dt * 1e9)


def tune_batch(replicas, mcs: int = 4, stream=None, policies=BATCH_POLICIES, measure_fn=None) -> dict:
    """Times every policy on the replica set (L, p, q, seed[, ...]) and returns
    the record of the choice, with `shapes`: the (Bx, By) for each replica."""
    replicas = [tuple(r[:4]) for r in replicas]
    fn = measure_fn or (lambda reps: measure_batch(reps, mcs, stream))
    table = []
    for pol in policies:
        reps = [r + batch_shape(int(r[0]), pol) for r in replicas]
        table.append({"policy": pol, "attempts_per_ns": float(fn(reps))})
    best = max(table, key=lambda row: row["attempts_per_ns"])
    return {"device": device_name() if measure_fn is None else "test", "key": batch_key(replicas),
            "policy": best["policy"], "attempts_per_ns": best["attempts_per_ns"], "table": table,
            "shapes": [batch_shape(int(r[0]), best["policy"]) for r in replicas], "mcs": mcs,
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


def choose_batch(replicas, cache: TuneCache | None = None, **kw) -> dict:
    """The recorded policy for this replica mix on this GPU, measuring once if there is none."""
    cache = cache if cache is not None else TuneCache()
    dev = device_name() if kw.get("measure_fn") is None else "test"
    key = f"{dev}|batch|{batch_key(replicas)}"
    rec = cache.entries.get(key)
    if rec is None:
        rec = tune_batch(replicas, **kw)
        cache.put_key(key, rec)
    return rec
