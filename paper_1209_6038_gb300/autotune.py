"""Autotuner of the integration schedule: the packet size (threads per block of the persistent kernel) and
the step-schedule knobs of cloak_set_schedule_tuning -- how many blocks take the slowest rays first, how
many rays they reserve per thread, and the resolution of the sort's cost buckets.  None of them changes a
result, only the time.

A coordinate search: starting from the handle's defaults, each knob in turn is set to each of its
candidates, the caller's render function is run once to warm up (and, for batches, to capture the CUDA
graph) and then timed with CUDA events; the fastest value is kept before the next knob is searched.  The
chosen schedule is left on the handle and cached per GPU and workload key in a JSON file next to this
module (_autotune.json, not versioned).
"""
from __future__ import annotations

import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")
CANDIDATES = (32, 64, 96, 128)  # threads per block of the persistent kernel (at most 128)
DEFAULT_SCHEDULE = {"packet": 128, "long_ray_blocks": 4, "reserve_per_thread": 1, "cost_scale": 4.0}
# the library's defaults for the mixed precisions (CLOAK_MIXED, CLOAK_MIXED_FF) while no schedule is set
MIXED_SCHEDULE = {"packet": 64, "long_ray_blocks": 16, "reserve_per_thread": 4, "cost_scale": 3.0}
SEARCH = (("packet", CANDIDATES), ("long_ray_blocks", (0, 2, 4, 8, 16)), ("cost_scale", (2.0, 3.0, 4.0, 6.0, 8.0)),
          ("reserve_per_thread", (1, 2, 4)))


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(full_key, entry):
    cache = _load()
    cache[full_key] = entry
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass


def _time(run, reps):
    import torch
    run()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return min(ms)


def apply(cloak, sched: dict):
    """Set a schedule (a dict with the keys of DEFAULT_SCHEDULE) on a wavefront handle."""
    from . import cloak as ck
    cloak.schedule(ck.SCHED_WAVEFRONT, int(sched["packet"]))
    ck.cloak_set_schedule_tuning(cloak.h, int(sched["long_ray_blocks"]), int(sched["reserve_per_thread"]),
                                 float(sched["cost_scale"]))


def tune_schedule(cloak, run, key: str, reps: int = 1, use_cache: bool = True, search=SEARCH, timer=None,
                  setter=None, device_name=None, start=None):
    """cloak: paper_1209_6038_gb300.cloak.Cloak (wavefront schedule); run(): one render on the current
    stream.  Returns (best schedule, {"knob=value": ms}).  The best schedule is left set on the handle.
    start: the schedule the search begins from (DEFAULT_SCHEDULE if None; MIXED_SCHEDULE suits the mixed
    precisions).  timer(run, reps) -> ms, setter(cloak, schedule) and device_name replace the CUDA-event
    timing, the handle call and the GPU's name (the search itself is host logic, tested without a GPU)."""
    timer = timer or _time
    setter = setter or apply
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    full_key = f"{device_name}|schedule|{key}"
    if use_cache:
        hit = _load().get(full_key)
        if hit:
            setter(cloak, hit["schedule"])
            return hit["schedule"], hit["ms"]
    best = dict(start or DEFAULT_SCHEDULE)
    setter(cloak, best)
    times = {"default": timer(run, reps)}
    best_ms = times["default"]
    for knob, values in search:
        incumbent = best[knob]  # already timed
        for v in values:
            if v == incumbent:
                continue
            trial = dict(best, **{knob: v})
            setter(cloak, trial)
            ms = timer(run, reps)
            times[f"{knob}={v}"] = ms
            if ms < best_ms:
                best_ms, best = ms, trial
        setter(cloak, best)
    _store(full_key, {"schedule": best, "ms": times})
    return best, times


def tune_packet(cloak, run, key: str, candidates=CANDIDATES, reps: int = 1, use_cache: bool = True):
    """The packet size alone (the other knobs at their defaults).  Returns (best_packet, {packet: ms})."""
    best, times = tune_schedule(cloak, run, f"packet|{key}", reps, use_cache, search=(("packet", candidates),))
    ms = {int(k.split("=")[1]): v for k, v in times.items() if k.startswith("packet=")}
    ms[DEFAULT_SCHEDULE["packet"]] = times["default"]
    return best["packet"], ms
