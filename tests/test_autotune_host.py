"""Host logic of the schedule autotuner (paper_1209_6038_gb300/autotune.py): the coordinate search over
the packet size and the step-schedule knobs, and its per-GPU cache, with a synthetic cost in place of the
timed batched render (no GPU)."""
import json

import pytest

from paper_1209_6038_gb300 import autotune


class FakeHandle:
    def __init__(self):
        self.schedule = None
        self.history = []


def setter(h, sched):
    h.schedule = dict(sched)
    h.history.append(dict(sched))


def make_timer(h, cost):
    calls = []

    def timer(run, reps):
        run()
        calls.append(dict(h.schedule))
        return cost(h.schedule)
    return timer, calls


def cost_a(s):
    # separable cost with its minimum at packet 64, 8 long-ray blocks, scale 3, 2 reserved rays
    return (abs(s["packet"] - 64) / 32 + abs(s["long_ray_blocks"] - 8) / 4 + abs(s["cost_scale"] - 3.0)
            + abs(s["reserve_per_thread"] - 2) + 100.0)


@pytest.fixture
def cache(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setattr(autotune, "CACHE", str(path))
    return path


def test_coordinate_search_finds_the_separable_minimum(cache):
    h = FakeHandle()
    timer, calls = make_timer(h, cost_a)
    runs = []
    best, times = autotune.tune_schedule(h, lambda: runs.append(1), "k", timer=timer, setter=setter,
                                         device_name="fake")
    assert best == {"packet": 64, "long_ray_blocks": 8, "reserve_per_thread": 2, "cost_scale": 3.0}
    assert h.schedule == best  # the chosen schedule is left on the handle
    # one timing of the default and one per candidate that differs from the current best
    n_cand = sum(len([v for v in vals if v != autotune.DEFAULT_SCHEDULE[k]]) for k, vals in autotune.SEARCH)
    assert len(calls) == len(runs) == 1 + n_cand == len(times)
    assert times["default"] == cost_a(autotune.DEFAULT_SCHEDULE)
    stored = json.loads(cache.read_text())
    assert stored["fake|schedule|k"]["schedule"] == best


def test_ties_keep_the_current_setting(cache):
    h = FakeHandle()
    timer, _ = make_timer(h, lambda s: 1.0)
    best, _ = autotune.tune_schedule(h, lambda: None, "flat", timer=timer, setter=setter, device_name="fake")
    assert best == autotune.DEFAULT_SCHEDULE


def test_cache_hit_skips_the_search_and_is_per_device(cache):
    h = FakeHandle()
    timer, calls = make_timer(h, cost_a)
    autotune.tune_schedule(h, lambda: None, "k", timer=timer, setter=setter, device_name="gpu A")
    n = len(calls)
    best, _ = autotune.tune_schedule(h, lambda: None, "k", timer=timer, setter=setter, device_name="gpu A")
    assert len(calls) == n and h.schedule == best
    autotune.tune_schedule(h, lambda: None, "k", timer=timer, setter=setter, device_name="gpu B")
    assert len(calls) > n  # another device tunes again
    h2 = FakeHandle()
    timer2, calls2 = make_timer(h2, cost_a)
    autotune.tune_schedule(h2, lambda: None, "k", timer=timer2, setter=setter, device_name="gpu A",
                           use_cache=False)
    assert len(calls2) == n  # use_cache=False searches again


def test_search_starts_from_the_given_schedule(cache):
    h = FakeHandle()
    timer, calls = make_timer(h, lambda s: 1.0)
    best, times = autotune.tune_schedule(h, lambda: None, "mixed", timer=timer, setter=setter, device_name="fake",
                                         start=autotune.MIXED_SCHEDULE)
    assert h.history[0] == autotune.MIXED_SCHEDULE and calls[0] == autotune.MIXED_SCHEDULE
    assert best == autotune.MIXED_SCHEDULE  # a flat cost keeps the start
    n_cand = sum(len([v for v in vals if v != autotune.MIXED_SCHEDULE[k]]) for k, vals in autotune.SEARCH)
    assert len(times) == 1 + n_cand
    # every start value is one of the search's candidates, so the search can come back to it
    for k, vals in autotune.SEARCH:
        assert autotune.MIXED_SCHEDULE[k] in vals and autotune.DEFAULT_SCHEDULE[k] in vals
