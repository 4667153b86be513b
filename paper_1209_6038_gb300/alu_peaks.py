"""Measured FP64 and FP32 FMA throughput of the GPU: the denominators of the ALU rooflines.

Runs the library's FMA microbenchmark (cloak_fma_peak: independent fused multiply-add chains, no memory
traffic) for a given wall time per precision on one GPU, timed with CUDA events on the launching stream,
while nvidia-smi samples the SM clocks.  Nothing here changes a clock or any other GPU setting.

  python -m paper_1209_6038_gb300.alu_peaks [--seconds S] [--out profiles/alu_peaks.json]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEFAULT_OUT = os.path.join(ROOT, "profiles", "alu_peaks.json")
BLOCKS_PER_SM, THREADS = 8, 256


def measure(seconds: float = 2.0, repeats: int = 3) -> dict:
    """Best-of-`repeats` FMA throughput (TFLOP/s) of FP64 and FP32 launches of about `seconds` each."""
    import torch

    from . import cloak as ck
    ck.load()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = BLOCKS_PER_SM * sms
    stream = torch.cuda.current_stream()
    out = {"sms": sms, "blocks": blocks, "threads": THREADS, "chains_per_thread": 8}
    for key, prec, dt in (("fp64", ck.FP64, torch.float64), ("fp32", ck.MIXED, torch.float32)):
        sink = torch.zeros(blocks * THREADS, dtype=dt, device="cuda")

        def run(iters):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            flops = ck.cloak_fma_peak(prec, blocks, THREADS, iters, sink)
            b.record(stream)
            b.synchronize()
            return flops, a.elapsed_time(b) / 1e3

        run(64)  # warm-up (module load)
        iters = 256
        while True:  # grow the launch until it runs for a tenth of the target time
            flops, t = run(iters)
            if t >= 0.1 * seconds or iters > (1 << 40):
                break
            iters *= 4
        iters = max(1, int(iters * seconds / max(t, 1e-6)))
        best = 0.0
        durations = []
        for _ in range(repeats):
            flops, t = run(iters)
            durations.append(t)
            best = max(best, flops / t / 1e12)
        out[key] = {"tflops": best, "iters": iters, "seconds": durations}
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=2.0)
    ap.add_argument("--repeats", type=int, default=3)
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args(argv)
    import torch

    from .clocks import ClockSampler
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    with sampler:
        res = measure(args.seconds, args.repeats)
    res["clocks"] = sampler.summary()
    res["gpu"] = torch.cuda.get_device_name(0)
    res["when"] = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    res["how"] = ("cloak_fma_peak: 8 blocks x 256 threads per SM, 8 independent FMA chains per thread, 2 flop per "
                  "FMA; CUDA events on the launching stream; best of the repeats")
    res["command"] = f"python -m paper_1209_6038_gb300.alu_peaks --seconds {args.seconds} --repeats {args.repeats}"
    if args.out:
        os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
            f.write("\n")
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
