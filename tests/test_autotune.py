"""Autotuner host logic (no GPU): candidate schedules, choice, cache."""
import json

import pytest

from paper_2407_01654_gb300 import autotune
from paper_2407_01654_gb300 import workloads as wl


def test_candidates_cover_both_loops_and_fitting_tile_heights():
    c = autotune.candidates(wl.make_params(nx=100, ny=20))
    assert c[0] == {"poisson_loop": 1, "tile_rows": 0}
    res = [x["tile_rows"] for x in c if x["poisson_loop"] == 2]
    assert res == [0, 8, 16, 24]  # heights up to the first one covering all 20 rows
    assert [x["tile_rows"] for x in c if x["poisson_loop"] == 3] == [0, 24]
    assert [x["tile_rows"] for x in c if x["poisson_loop"] == 4] == [0]
    c = autotune.candidates(wl.make_params(nx=512, ny=1024))
    assert [x["tile_rows"] for x in c if x["poisson_loop"] == 2] == [0, 8, 16, 24, 32, 40, 48, 56, 64]
    assert [x["tile_rows"] for x in c if x["poisson_loop"] == 3] == [0, 24, 32, 40, 48, 56, 64]
    assert [x["tile_rows"] for x in c if x["poisson_loop"] == 4] == [0, 48, 56, 64]


def test_pick_fastest_skips_failures_and_keeps_first_on_ties():
    a, b, c = {"k": 1}, {"k": 2}, {"k": 3}
    assert autotune.pick([(a, 2.0), (b, None), (c, 1.0)]) == (c, 1.0)
    assert autotune.pick([(a, 1.0), (b, 1.0)]) == (a, 1.0)
    with pytest.raises(RuntimeError):
        autotune.pick([(a, None), (b, float("nan"))])


def test_tune_times_every_candidate_once_then_uses_the_cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("EHD_AUTOTUNE_CACHE", str(path))
    p = wl.make_params(nx=128, ny=64)
    calls = []

    def fake(params, fields, ov, steps, fixed_iter):
        calls.append(ov)
        assert fixed_iter > 0 and fields["phi"].shape == (64, 128)
        return 1.0 if ov["poisson_loop"] == 1 else 0.5 + abs(ov["tile_rows"] - 32) / 100

    best = autotune.tune(p, timer=fake, device_name="dev")
    assert best == {"poisson_loop": 2, "tile_rows": 32}
    assert len(calls) == len(autotune.candidates(p))
    d = json.loads(path.read_text())
    assert d["dev|128x64|walls1|prec0"]["overrides"] == best
    calls.clear()
    assert autotune.tune(p, timer=fake, device_name="dev") == best
    assert calls == []                       # served from the cache
    assert autotune.tune(p, timer=fake, device_name="other") == best
    assert len(calls) == len(autotune.candidates(p))  # another device tunes again


def test_tune_batch_picks_the_highest_rate_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("EHD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    reqs = [(wl.make_params(nx=64, ny=64), {}), (wl.make_params(nx=128, ny=128), {})]
    calls = []

    def fake(requests, schedule, steps, budget):
        calls.append(schedule)
        if schedule["tile_rows"] == 64:
            return None                       # nothing admitted
        return 1e9 * (2 if schedule == {"tile_rows": 16, "steps_per_graph": 32} else 1)

    best = autotune.tune_batch(reqs, timer=fake, device_name="dev")
    assert best == {"tile_rows": 16, "steps_per_graph": 32}
    assert len(calls) == len(autotune.batch_candidates()) == 9
    calls.clear()
    assert autotune.tune_batch(list(reversed(reqs)), timer=fake, device_name="dev") == best
    assert calls == []                        # same mix of shapes: from the cache
