"""Autotuner for the packet size (threads per block) of the persistent integration kernel.

Each candidate is set on the handle (cloak_set_schedule), the caller's render function is run once to
warm up (and, for batches, to capture the CUDA graph) and then timed with CUDA events; the fastest
candidate is kept on the handle and cached per GPU and workload key in a JSON file next to this
module (_autotune.json, not versioned).
"""
from __future__ import annotations

import json
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")
CANDIDATES = (32, 64, 96, 128)  # threads per block of the persistent kernel (at most 128)


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune_packet(cloak, run, key: str, candidates=CANDIDATES, reps: int = 1, use_cache: bool = True):
    """cloak: paper_1209_6038_gb300.cloak.Cloak (wavefront schedule); run(): one render on the current
    stream.  Returns (best_packet, {packet: ms}).  The best packet is left set on the handle."""
    import torch
    from . import cloak as ck
    gpu = torch.cuda.get_device_name()
    full_key = f"{gpu}|{key}"
    cache = _load()
    if use_cache and full_key in cache:
        best = int(cache[full_key]["packet"])
        cloak.schedule(ck.SCHED_WAVEFRONT, best)
        return best, cache[full_key]["ms"]
    times = {}
    for pk in candidates:
        cloak.schedule(ck.SCHED_WAVEFRONT, pk)
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
        times[pk] = min(ms)
    best = min(times, key=times.get)
    cloak.schedule(ck.SCHED_WAVEFRONT, best)
    cache[full_key] = {"packet": best, "ms": {str(k): v for k, v in times.items()}}
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return best, times
