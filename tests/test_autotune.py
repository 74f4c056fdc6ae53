"""Host logic of the block-tile autotuner (no GPU): candidate shapes, the
choice, and the record that makes a tuned run reproducible."""
import json

import pytest

from paper_1705_01022_gb300 import autotune as at


@pytest.mark.parametrize("L", [64, 128, 192, 256, 1024, 4096, 131072])
def test_candidates_are_valid_shapes(L):
    shapes = at.candidates(L)
    assert shapes, L
    for Bx, By in shapes:
        gx, gy = Bx // 32, By // 16
        assert Bx % 32 == 0 and By % 16 == 0
        assert gx * gy <= 32
        assert gx & (gx - 1) == 0 and gy & (gy - 1) == 0
        assert L % (2 * Bx) == 0 and L % (2 * By) == 0
    assert len(set(shapes)) == len(shapes)


def test_candidates_at_the_bench_size():
    shapes = at.candidates(1 << 17)
    assert (256, 64) in shapes
    # every split of 32 groups into powers of two, down to one group
    assert len(shapes) == 21
    assert shapes[0][0] * shapes[0][1] == 32 * 32 * 16


def test_non_power_of_two_groups_when_asked():
    assert (96, 32) in at.candidates(192, pow2=False)
    assert (96, 32) not in at.candidates(192)


def test_mode():
    assert at.mode_of(1.0, 0.0) == "deterministic"
    assert at.mode_of(0.0, 1.0) == "deterministic"
    assert at.mode_of(0.95, 0.05) == "random"
    assert at.mode_of(1.0, 0.5) == "random"


def test_pick_fastest_and_deterministic_ties():
    table = [{"Bx": 256, "By": 64, "attempts_per_ns": 10.0},
             {"Bx": 128, "By": 128, "attempts_per_ns": 12.0},
             {"Bx": 64, "By": 256, "attempts_per_ns": 12.0}]
    assert (at.pick(table)["Bx"], at.pick(table)["By"]) == (128, 128)


def test_tune_with_a_fake_timer_and_cache_round_trip(tmp_path):
    calls = []

    def fake(Bx, By):
        calls.append((Bx, By))
        return 1000.0 - abs(Bx - 256) - abs(By - 64)

    path = str(tmp_path / "tune.json")
    cache = at.TuneCache.load(path)
    rec = at.choose(1 << 17, 0.95, 0.05, cache=cache, measure_fn=fake)
    assert (rec["Bx"], rec["By"]) == (256, 64)
    assert (rec["cx"], rec["cy"]) == at.CELL
    assert len(rec["table"]) == len(at.candidates(1 << 17)) == len(calls)
    # recorded: a second lookup (fresh cache object from the file) does not measure again
    calls.clear()
    again = at.choose(1 << 17, 0.95, 0.05, cache=at.TuneCache.load(path), measure_fn=fake)
    assert calls == [] and (again["Bx"], again["By"]) == (256, 64)
    with open(path) as f:
        stored = json.load(f)
    assert list(stored) == [at.TuneCache.key("test", 1 << 17, "random")]
    # another acceptance mode is a separate decision
    at.choose(1 << 17, 1.0, 0.0, cache=cache, measure_fn=fake)
    assert len(at.TuneCache.load(path).entries) == 2


def test_no_shape_fits():
    with pytest.raises(ValueError):
        at.tune(96, 1.0, 0.0, measure_fn=lambda Bx, By: 1.0)


def test_batch_policies_give_valid_shapes():
    for L in range(64, 4097, 64):
        assert at.batch_shape(L, "default") == ((64, 64) if L % 128 == 0 else (32, 32))
        for pol in ("wide", "square"):
            Bx, By = at.batch_shape(L, pol)
            assert (Bx, By) in at.candidates(L)
            assert at.groups((Bx, By)) == max(at.groups(s) for s in at.candidates(L))
        Bx, By = at.batch_shape(L, "tall")
        assert (Bx, By) in at.candidates(L)
        if at.groups(at.batch_shape(L, "wide")) == at.MAX_GROUPS:
            assert (Bx, By) == at.batch_shape(L, "wide")
        else:
            assert Bx == 32 and By == max(s[1] for s in at.candidates(L) if s[0] == 32)
    assert at.batch_shape(4096, "wide") == (1024, 16)
    assert at.batch_shape(4096, "square") == (128, 128)
    assert at.batch_shape(192, "wide") == (32, 32)
    assert at.batch_shape(384, "wide") == (64, 64) and at.batch_shape(384, "tall") == (32, 64)
    # 'large': full-warp sub-tiles only where they leave enough of them per device step
    assert at.batch_shape(4096, "large") == (64, 64)
    assert at.batch_shape(6144, "large") == (64, 64)
    assert at.batch_shape(8192, "large") == (1024, 16)
    assert at.batch_shape(16384, "large") == (1024, 16)
    for L in range(128, 16385, 128):
        Bx, By = at.batch_shape(L, "large")
        assert (Bx, By) in at.candidates(L) or (Bx, By) == at.batch_shape(L, "default")


def test_tune_batch_with_a_fake_timer(tmp_path):
    reps = [(L, p, q, 100 + i) for i, (L, (p, q)) in
            enumerate(zip(range(64, 4097, 64), [(1.0, 0.0), (0.95, 0.05), (0.5, 0.5)] * 30))]
    seen = []

    def fake(rs):
        seen.append(rs)
        return {(64, 64): 900.0}.get(rs[-1][4:], 1000.0) if rs[-1][4:] != (128, 128) else 1100.0

    cache = at.TuneCache.load(str(tmp_path / "b.json"))
    rec = at.choose_batch(reps, cache=cache, measure_fn=fake)
    assert rec["policy"] == "square" and len(rec["shapes"]) == len(reps)
    assert [row["policy"] for row in rec["table"]] == list(at.BATCH_POLICIES)
    assert all(len(r) == 6 for r in seen[0])
    seen.clear()
    again = at.choose_batch(reps, cache=at.TuneCache.load(cache.path), measure_fn=fake)
    assert seen == [] and again["policy"] == "square"
    # a different mix is a different decision
    assert at.batch_key(reps) != at.batch_key(reps[:-1])


# ------------------------------------------------------------ thread cell ---

def test_cells_are_the_supported_shapes_finest_first():
    areas = [cx * cy for cx, cy in at.CELLS]
    assert areas == sorted(areas) and at.CELLS[0] == (4, 4) and at.CELLS[-1] == (32, 16)
    assert len(set(at.CELLS)) == len(at.CELLS)
    for cx, cy in at.CELLS:
        assert cx in (4, 8, 16, 32) and cy in (4, 8, 16)


def test_relative_w2_of_independent_ensembles():
    a = [[2.0, 4.0], [4.0, 8.0]]
    b = [[3.0, 6.0], [3.0, 6.0]]
    rel = at.relative_w2(a, b)
    assert rel[0][0] == pytest.approx(1.0) and rel[1][0] == pytest.approx(1.0)
    # var(a)/n = 2/2 = 1 at t0, mean 3: error = 1 * sqrt(1/9)
    assert rel[0][1] == pytest.approx(1.0 / 3.0)
    assert at.relative_w2([[1.0], [1.0]], [[2.0], [2.0]]) == [(0.5, 0.0)]


def _fake_cells(shift_per_area):
    """Rates fall with the cell's area, the W^2 deficit falls with it too."""
    def rate(c):
        return 2000.0 * 16 / (c[0] * c[1])

    def w2(c):
        d = shift_per_area / (c[0] * c[1])
        return [[10.0 * (1 - d), 20.0 * (1 - d)], [10.0 * (1 - d), 20.0 * (1 - d)]]
    return rate, w2


@pytest.mark.parametrize("max_shift,want", [(0.0, (32, 16)), (0.003, (16, 16)), (0.005, (16, 8)),
                                            (0.02, (8, 4)), (0.05, (4, 4))])
def test_fastest_cell_within_the_allowed_shift(max_shift, want):
    # deficit 0.64/area against exact W^2: 4x4 4 %, 8x4 2 %, 8x8 1 %, 16x8 0.5 %, 16x16 0.25 %, 32x16
    # 0.125 %; relative to 32x16 that is a shift of 3.9 %, 1.9 %, 0.88 %, 0.38 % and 0.13 %; equal rates
    # (16x16 and 32x8) go to the first in CELLS
    rate, w2 = _fake_cells(0.64)
    rec = at.tune_cell(4096, 1.0, 0.0, 256, 64, max_shift=max_shift, measure_fn=rate, w2_fn=w2)
    assert (rec["cx"], rec["cy"]) == want
    assert rec["reference"] == [32, 16]
    ref_row = [r for r in rec["table"] if (r["cx"], r["cy"]) == (32, 16)][0]
    assert ref_row["w2_ratio"] == [1.0, 1.0]
    assert len(rec["table"]) == len(at.CELLS)
    chosen = [r for r in rec["table"] if (r["cx"], r["cy"]) == want][0]
    assert rec["attempts_per_ns"] == chosen["attempts_per_ns"]


def test_cell_choice_is_recorded_and_reused(tmp_path):
    rate, w2 = _fake_cells(0.64)
    calls = []

    def counting_rate(c):
        calls.append(c)
        return rate(c)

    path = str(tmp_path / "tune.json")
    rec = at.choose_cell(1 << 17, 0.95, 0.05, 256, 64, max_shift=0.02, cache=at.TuneCache.load(path),
                         measure_fn=counting_rate, w2_fn=w2)
    assert len(calls) == len(at.CELLS)
    calls.clear()
    again = at.choose_cell(1 << 17, 0.95, 0.05, 256, 64, max_shift=0.02, cache=at.TuneCache.load(path),
                           measure_fn=counting_rate, w2_fn=w2)
    assert calls == [] and (again["cx"], again["cy"]) == (rec["cx"], rec["cy"]) and again["when"] == rec["when"]
    # another tolerance or another (p, q) is a separate decision
    at.choose_cell(1 << 17, 0.95, 0.05, 256, 64, max_shift=0.001, cache=at.TuneCache.load(path),
                   measure_fn=counting_rate, w2_fn=w2)
    at.choose_cell(1 << 17, 0.5, 0.5, 256, 64, max_shift=0.02, cache=at.TuneCache.load(path),
                   measure_fn=counting_rate, w2_fn=w2)
    assert len(at.TuneCache.load(path).entries) == 3


def test_reference_cell_is_chosen_when_every_finer_cell_shifts_too_much():
    rate, w2 = _fake_cells(50.0)
    rec = at.tune_cell(1024, 0.5, 0.5, 64, 64, max_shift=0.01, measure_fn=rate, w2_fn=w2,
                       cells=[(4, 4), (8, 8), (16, 16)])
    assert (rec["cx"], rec["cy"]) == (16, 16) and rec["reference"] == [16, 16]
