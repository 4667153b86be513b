#!/usr/bin/env python
"""Benchmark of the uniaxial-cloak renderer on one node.

A step renders every image of the full workload: radial and azimuthal cloaks
(Eqs. 14, 15) x ordinary and extraordinary light x camera elevations 0/20/45 deg,
1920x1080 pixels, 4 jittered samples per pixel, Dormand-Prince 5(4) at tolerance
1e-9 in FP64 -- 99.5 million camera rays.  The value is traced camera rays per
second (whole job).  Also reported: the plain FP64 path (one thread per pixel),
the roofline of the dominant kernel against the FP64 ALU peak, the CPU FP64
oracle on a bounded sample of the same workload (and the exit-direction error
against it), an end-to-end number through the public API with the images copied
to pinned host memory, the SM clocks seen during the timed region, the mixed-
precision forms (the band near R1 in FP64 and in double-float) with their error
against the oracle, the learned surrogate with its FP64 fallback, a 256-view
batched orbit and the Fermat/Hamiltonian comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "traced rays/s at 1920x1080 vs plain FP64 GPU integrator; max exit-dir err"
UNIT = "rays/s"

# FP64 and FP32 ALU peaks: FMA throughput measured on this GPU model by the library's microbenchmark
# (paper_1209_6038_gb300/alu_peaks.py: independent FMA chains, CUDA events, clocks sampled), committed in
# profiles/alu_peaks.json; the bench re-measures them for a second each and reports both.  Without the file
# the unit-count derivation stands in (152 SMs x 2070 MHz x 4 FP64 / 256 FP32 flop per clock per SM).
ALU_PEAKS_PATH = os.path.join(ROOT, "profiles", "alu_peaks.json")


def _alu_peaks():
    try:
        with open(ALU_PEAKS_PATH) as f:
            d = json.load(f)
        return (float(d["fp64"]["tflops"]), float(d["fp32"]["tflops"]),
                f"measured: FMA microbenchmark, profiles/alu_peaks.json ({d.get('gpu', 'GPU')}, "
                f"SM {d.get('clocks', {}).get('sm_mhz')} MHz)")
    except (OSError, ValueError, KeyError):
        return 152 * 2.070e9 * 4 / 1e12, 152 * 2.070e9 * 256 / 1e12, "derived: 152 SM x 2.07 GHz x 4 / 256 flop/clk/SM"


FP64_PEAK_TFLOPS, FP32_PEAK_TFLOPS, ALU_PEAK_SOURCE = _alu_peaks()


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# dense BF16 tensor peak: measured on the GB300s (cuBLAS, burst; sustained for a seconds-long
# loop), else the recipe's fallback
BF16_PEAK_TFLOPS = float(_measured_peaks().get("bf16_tflops", 1900.0))
BF16_PEAK_SUSTAINED_TFLOPS = float(_measured_peaks().get("bf16_tflops_sustained", 1700.0))

# Algorithmic FP64 flops per integrator step attempt, counted from the source formulas
# (FMA = 2 flops, reciprocal and 1/sqrt = 1 flop each):
#   RHS of Eq. 8 / Eq. 2 in closed cylindrical form: radial-e 36, azimuthal-e 30,
#   azimuthal-o 34, radial-o 0 (straight lines, Sect. 4).
#   DP5(4) attempt: 6 new RHS + stage combinations as FMA chains on h-scaled coefficients (332) + error
#   norm (30).
#   RK4 step: 4 RHS + combinations (102).
RHS_FLOPS = {(0, 0): 0, (0, 1): 36, (1, 0): 34, (1, 1): 30}

# DRAM bytes (read + write) of one launch of the any-medium integration kernel on the full step: one
# ncu capture of the same twelve views at 480x270 x 4 spp (122.5 MB read + 54.1 MB written) scaled by
# samples (x 16.0).  To be re-captured whenever the kernel changes.
INTEGRATE_TRAFFIC_BYTES = (122.350336e6 + 54.126080e6) * (1920 * 1080) / (480 * 270)
DP45_FIXED, RK4_FIXED = 362, 102

# bytes per view of the table a batched render copies host to device at every step (the camera frame,
# sample offsets, output pointer and size of each view; csrc/batch.h: ViewDev)
VIEW_TABLE_BYTES = 152


def flops_per_step(variant, mode, integ):
    r = RHS_FLOPS[(variant, mode)]
    return 6 * r + DP45_FIXED if integ == 1 else 4 * r + RK4_FIXED


from paper_1209_6038_gb300.clocks import ClockSampler  # noqa: E402


def dist_env():
    from paper_1209_6038_gb300.replicas import dist_env as env
    return env()


# ------------------------------------------------------------------ reference arm (the CPU oracle)
def sample_pixels(w, img_index, n, seed=12345):
    from paper_1209_6038_gb300 import inputs
    return inputs.sample_pixels(w, img_index, n, seed)


def run_oracle_sample(w, pix_per_image, nthreads, seed=12345):
    """The CPU FP64 oracle on a seeded pixel sample of every image; returns (rays, seconds, records)."""
    import oracle as O
    from paper_1209_6038_gb300 import inputs
    recs = []
    t0 = time.perf_counter()
    for idx, (v, m, e) in enumerate(w.images):
        eye, tgt, up = inputs.camera_pose(e)
        pix = sample_pixels(w, idx, pix_per_image, seed)
        integ = O.Integrator(O.DP45 if w.integrator == "dp45" else O.RK4, w.h_or_tol, w.max_steps)
        _, rec = O.render(O.Cloak(v), integ, O.Camera(eye, tgt, up, w.hfov_deg, w.width, w.height), m, w.spp,
                          w.seed, pixels=pix, nthreads=nthreads)
        recs.append(rec)
    dt = time.perf_counter() - t0
    return pix_per_image * w.spp * len(w.images), dt, recs


GOLDEN = os.path.join(ROOT, "tests", "golden")


def angles(a, b):
    import numpy as np
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cr, np.sum(a * b, axis=-1))


def _golden_rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def _sample_positions(w, npix):
    """flat sample index -> position in the concatenated oracle sample, per image"""
    import numpy as np
    pos = []
    off = 0
    for idx in range(len(w.images)):
        pix = sample_pixels(w, idx, npix)
        samp = (pix[:, None] * w.spp + np.arange(w.spp)[None, :]).reshape(-1)
        pos.append({int(s): off + k for k, s in enumerate(samp)})
        off += len(samp)
    return pos


def reference_records(w, o, npix):
    """The FP64 oracle's records of the benchmark sample with the binary128 reference in place of the rays the
    FP64 oracle does not determine; per-ray FP64 bars (1e-9 + 8 D64) and the mask of those rays."""
    import numpy as np
    ref = o.copy()
    lim = np.full(len(ref), 1e-9)
    und = np.zeros(len(ref), bool)
    if npix != 100000:  # the stored reference belongs to the 100000-pixel sample
        return ref, lim, und
    pos = _sample_positions(w, npix)
    for f in _golden_rows("fp64_undetermined_rays.txt"):
        k = pos[int(f[0])][int(f[1])]
        ref["status"][k], ref["steps"][k] = int(f[2]), int(f[3])
        ref["exit_dir"][k] = [float(x) for x in f[4:7]]
        ref["exit_pos"][k] = [float(x) for x in f[7:10]]
        ref["tof"][k], ref["weight"][k], ref["tile_id"][k] = float(f[10]), float(f[11]), int(f[12])
        lim[k] = 1e-9 + 8.0 * max(float(x) for x in f[16:19])
        und[k] = True
    return ref, lim, und


def fp32_bars(w, npix):
    """Per-ray exit-direction bars of the mixed path on the benchmark sample, min(1e-4, max(1e-5, 100 D32)) with D32
    the distance an FP32 model of the oracle moves the ray, and the statuses FP32 does not fix."""
    import numpy as np
    n = len(w.images) * npix * w.spp
    lim = np.full(n, 1e-5)
    flip = np.zeros(n, bool)
    if npix != 100000:
        return lim, flip
    pos = _sample_positions(w, npix)
    for f in _golden_rows("fp32_sensitive_rays.txt"):
        k = pos[int(f[0])][int(f[1])]
        d32 = float(f[2])
        if d32 > 1e-7:
            lim[k] = min(1e-4, 100.0 * d32)
        flip[k] = f[3] == "1"
    return lim, flip


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import build as obuild
    obuild.build()
    from paper_1209_6038_gb300 import inputs
    w = inputs.FULL
    cores = os.cpu_count() or 1
    per_image = args.ref_pixels
    for _ in range(args.warmup):
        run_oracle_sample(w, max(8, per_image // 8), cores, seed=999)
    times, nrays = [], 0
    for k in range(args.steps):
        n, dt, _ = run_oracle_sample(w, per_image, cores, seed=12345 + 100 * k)
        times.append(dt)
        nrays += n
    total = sum(times)
    value = nrays / total
    sample = (f"{per_image} seeded pixels x {w.spp} spp from each of the {len(w.images)} images per step "
              f"({per_image * w.spp * len(w.images)} rays/step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(w):
    return {"workload": w.name, "width": w.width, "height": w.height, "spp": w.spp,
            "images": len(w.images), "variants": ["radial", "azimuthal"][: len(w.variants)],
            "polarizations": ["ordinary", "extraordinary"][: len(w.pols)], "elevations_deg": list(w.elevations),
            "integrator": w.integrator, "tol": w.h_or_tol, "camera_distance": 5.0, "hfov_deg": w.hfov_deg,
            "geometry": {"R1": 0.5, "R2": 1.0, "height": 2.0}, "scene": "procedural checkerboard room, seed 0",
            "parallelism": "one process per GPU, every rank renders the full workload (replicas)",
            "l2": "256 MiB buffer written between timed steps"}


# ------------------------------------------------------------------ learned surrogate
SUR_FLOPS_PER_RAY = 2 * (7 * 256 + 3 * 256 * 256 + 256 * 5)  # algorithmic multiply-adds x 2 of one forward pass


def surrogate_section(args, ck, inputs, torch, np, flush):
    """Train the surrogate once on rays traced by the FP64 integrator, then render the views of the
    surrogate workload with it (integrator fallback) and with the FP64 integrator alone, each as one
    batched render of all views: rays/s of both, the share of rays the surrogate finished, the image error
    against the FP64 integrator (per-view records), and the tensor-core roofline of the network's forward
    pass."""
    sw = inputs.SURROGATE
    integ = ck.DP45 if sw.integrator == "dp45" else ck.RK4
    trainer = ck.Cloak(ck.RADIAL).integrator(integ, sw.h_or_tol, ck.FP64, sw.max_steps)
    t0 = time.perf_counter()
    ck.cloak_surrogate_train(trainer.h, sw.extra["train_rays"], sw.extra["train_seed"], args.sur_epochs)
    train_wall = time.perf_counter() - t0
    info = ck.cloak_surrogate_info(trainer.h)
    tt = ck.cloak_surrogate_train_timing(trainer.h)
    train_tflops = tt["flops_per_step_stage1"] / (tt["ms_per_step_stage1"] / 1e3) / 1e12
    path = os.path.join(tempfile.gettempdir(), f"cloak_surrogate_{os.getpid()}.bin")
    ck.cloak_surrogate_save(trainer.h, path)
    # reproducibility: the same seed trains the same network (fixed-order gradient sums), bit for bit; other
    # seeds give the run-to-run spread of what the network takes over
    params0 = ck.cloak_surrogate_params(trainer.h)
    rb_small = torch.empty(sw.rays_per_image * ck.RECORD_BYTES, dtype=torch.uint8, device="cuda")

    def handled_fraction(net_path, stride=49):
        """share of the entering rays (every stride-th sample of every view) the gate leaves to the network"""
        ent = hnd = 0
        for v, m, e in sw.images:
            eye, tgt, up = inputs.camera_pose(e)
            c = ck.Cloak(v).camera(eye, tgt, up, sw.hfov_deg, sw.width, sw.height)
            c.integrator(integ, sw.h_or_tol, ck.SURROGATE, sw.max_steps).schedule(ck.SCHED_WAVEFRONT)
            ck.cloak_surrogate_load(c.h, net_path)
            ck.cloak_surrogate_set_gate(c.h, sw.extra["gate_log10_err"])
            c.render_records(m, sw.spp, sw.seed, out=rb_small)
            r = ck.records_to_numpy(rb_small.view(-1, ck.RECORD_BYTES)[::stride].contiguous().reshape(-1))
            ent += int((r["status"] != 0).sum())
            hnd += int(((r["steps"] == 0) & np.isin(r["status"], [1, 2])).sum())
            c.close()
        return hnd / max(1, ent)

    shares = {"seed_0": handled_fraction(path)}
    again = ck.Cloak(ck.RADIAL).integrator(integ, sw.h_or_tol, ck.FP64, sw.max_steps)
    ck.cloak_surrogate_train(again.h, sw.extra["train_rays"], sw.extra["train_seed"], args.sur_epochs)
    same_seed_identical = bool(np.array_equal(ck.cloak_surrogate_params(again.h), params0))
    again.close()
    for sd in (1, 2):
        other = ck.Cloak(ck.RADIAL).integrator(integ, sw.h_or_tol, ck.FP64, sw.max_steps)
        ck.cloak_surrogate_train(other.h, sw.extra["train_rays"], sd, args.sur_epochs)
        op = os.path.join(tempfile.gettempdir(), f"cloak_surrogate_{os.getpid()}_{sd}.bin")
        ck.cloak_surrogate_save(other.h, op)
        other.close()
        shares[f"seed_{sd}"] = handled_fraction(op)
        os.remove(op)
    del rb_small
    # forward pass of 2^22 rows on the tensor cores (one fused persistent launch)
    n = 1 << 22
    x = torch.rand((n, 7), device="cuda") * 2 - 1
    y = torch.empty((n, 5), device="cuda")
    def fwd_time(fp16):
        ck.cloak_surrogate_set_precision(trainer.h, fp16)
        ck.cloak_surrogate_forward(trainer.h, x, y)
        ms = []
        for _ in range(5):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ck.cloak_surrogate_forward(trainer.h, x, y)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    fwd_ms16 = fwd_time(True)   # FP16 operands (optional inference precision)
    fwd_ms = fwd_time(False)    # BF16 operands, the training precision (default)
    achieved = n * SUR_FLOPS_PER_RAY / (fwd_ms / 1e3) / 1e12
    peak = BF16_PEAK_TFLOPS
    trainer.close()
    del x, y
    hs = {}
    for v in sw.variants:
        for prec in (ck.FP64, ck.SURROGATE):
            c = ck.Cloak(v).integrator(integ, sw.h_or_tol, prec, sw.max_steps).schedule(ck.SCHED_WAVEFRONT)
            if prec == ck.SURROGATE:
                ck.cloak_surrogate_load(c.h, path)
                ck.cloak_surrogate_set_gate(c.h, sw.extra["gate_log10_err"])
            hs[(v, prec)] = c
    # the timed renders: all views in one batched render (one queue, the network and gate on every queued
    # ray, one persistent integration launch for the rest), with the FP64 integrator alone for comparison
    bh = {}
    for prec in (ck.FP64, ck.SURROGATE):
        b = ck.Cloak(ck.RADIAL).integrator(integ, sw.h_or_tol, prec, sw.max_steps).schedule(ck.SCHED_WAVEFRONT)
        b.stage_timing(True)
        if prec == ck.SURROGATE:
            ck.cloak_surrogate_load(b.h, path)
            ck.cloak_surrogate_set_gate(b.h, sw.extra["gate_log10_err"])
        bh[prec] = b
    os.remove(path)
    bviews = []
    for v, m, e in sw.images:
        eye, tgt, up = inputs.camera_pose(e)
        bviews.append((v, m, eye, tgt, up, sw.hfov_deg,
                       torch.empty((sw.height, sw.width, 4), dtype=torch.float32, device="cuda")))

    def view(c, e):
        eye, tgt, up = inputs.camera_pose(e)
        c.camera(eye, tgt, up, sw.hfov_deg, sw.width, sw.height)

    def step(prec):
        ck.cloak_render_batch(bh[prec].h, bviews, sw.spp, sw.seed)

    def timed_render(prec):
        step(prec)
        torch.cuda.synchronize()
        st = list(bh[prec].stage_times())
        ts = []
        for _ in range(2):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step(prec)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts), st

    res, stages = {}, {}
    for prec in (ck.FP64, ck.SURROGATE):
        res[prec], stages[prec] = timed_render(prec)
    # the same surrogate render with FP16 inference
    ck.cloak_surrogate_set_precision(bh[ck.SURROGATE].h, True)
    res16, stages16 = timed_render(ck.SURROGATE)
    ck.cloak_surrogate_set_precision(bh[ck.SURROGATE].h, False)
    # image error against the FP64 integrator, ray by ray
    rb = torch.empty(sw.rays_per_image * ck.RECORD_BYTES, dtype=torch.uint8, device="cuda")
    tot = {"rays": 0, "entering": 0, "handled": 0, "tile_all": 0, "tile_cloak": 0, "status": 0}
    errs = []
    for v, m, e in sw.images:
        recs = []
        for prec in (ck.FP64, ck.SURROGATE):
            c = hs[(v, prec)]
            view(c, e)
            c.render_records(m, sw.spp, sw.seed, out=rb)
            # every 7th sample of the image (about 1.2 million rays per image)
            recs.append(ck.records_to_numpy(rb.view(-1, ck.RECORD_BYTES)[::7].contiguous().reshape(-1)))
        a, b = recs
        entering = a["status"] != 0
        handled = (b["steps"] == 0) & np.isin(b["status"], [1, 2])
        diff = a["tile_id"] != b["tile_id"]
        tot["rays"] += a.size
        tot["entering"] += int(entering.sum())
        tot["handled"] += int(handled.sum())
        tot["tile_all"] += int(diff.sum())
        tot["tile_cloak"] += int((diff & entering).sum())
        tot["status"] += int((a["status"] != b["status"]).sum())
        da, db = a["exit_dir"][handled], b["exit_dir"][handled]
        errs.append(np.arctan2(np.linalg.norm(np.cross(da, db), axis=-1), np.sum(da * db, axis=-1)))
    for c in list(hs.values()) + list(bh.values()):
        c.close()
    del bviews
    err = np.concatenate(errs)
    rays = sw.rays
    return {"workload": sw.name + ", one batched render of all views", "value": rays / (res[ck.SURROGATE] / 1e3),
            "unit": "rays/s",
            "ms_per_step": res[ck.SURROGATE], "fp64_integrator": {"value": rays / (res[ck.FP64] / 1e3),
                                                                   "ms_per_step": res[ck.FP64]},
            "speedup_vs_fp64_integrator": res[ck.FP64] / res[ck.SURROGATE], "warmup": 1, "steps": 2,
            "stage_ms": {name: {"surrogate": stages[ck.SURROGATE][k], "fp64_integrator": stages[ck.FP64][k]}
                         for k, name in enumerate(("camera_entry_network_gate_sort", "integrate", "exit_shade",
                                                   "resolve"))},
            "network_features_gate_ms": stages[ck.SURROGATE][0] - stages[ck.FP64][0],
            "fp16_inference": {"value": rays / (res16 / 1e3), "ms_per_step": res16,
                               "speedup_vs_fp64_integrator": res[ck.FP64] / res16,
                               "network_features_gate_ms": stages16[0] - stages[ck.FP64][0],
                               "forward_tflops": n * SUR_FLOPS_PER_RAY / (fwd_ms16 / 1e3) / 1e12,
                               "forward_frac_of_peak": n * SUR_FLOPS_PER_RAY / (fwd_ms16 / 1e3) / 1e12 / peak,
                               "note": "cloak_surrogate_set_precision(h, 1): FP16 weights, hidden biases, input "
                                       "pairs and activations, FP32 accumulation; same peak as BF16"},
            "gate_log10_err": sw.extra["gate_log10_err"],
            "handled_frac_of_entering": tot["handled"] / max(1, tot["entering"]),
            "image_error_vs_fp64": {"sample": "every 7th ray of every view", "rays_compared": tot["rays"],
                                    "tile_differs_frac": tot["tile_all"] / tot["rays"],
                                    "tile_differs_frac_of_cloak_rays": tot["tile_cloak"] / max(1, tot["entering"]),
                                    "status_differs_frac": tot["status"] / tot["rays"],
                                    "handled_exit_dir_err_rad": {"median": float(np.median(err)) if err.size else None,
                                                                 "p99": float(np.quantile(err, 0.99)) if err.size else None,
                                                                 "max": float(err.max()) if err.size else None}},
            "training": {**{k: float(v) for k, v in info.items()}, "wall_s": train_wall, "epochs": args.sur_epochs,
                         "same_seed_bit_identical": same_seed_identical,
                         "handled_frac_by_training_seed": shares,
                         "roofline": {"bound": "tensor", "achieved": train_tflops, "peak": BF16_PEAK_SUSTAINED_TFLOPS,
                                      "unit": "TFLOP/s", "frac": train_tflops / BF16_PEAK_SUSTAINED_TFLOPS,
                                      "ms_per_step": tt["ms_per_step_stage1"], "batch": tt["batch"],
                                      "flops_per_step": tt["flops_per_step_stage1"],
                                      "peak_source": "measured cuBLAS bf16 GEMM, sustained (MEASURED_PEAKS.json)",
                                      "note": "one stage-1 optimizer step: batch gather, forward, loss, backward "
                                              "(data and weight GEMMs, fixed-order split-K sums) and Adam, replayed "
                                              "as a CUDA graph; CUDA events around the stage"}},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst) of measured",
                         "kernel": "k_mlp_fused (persistent tcgen05 network, BF16 operands, FP32 accumulation in TMEM): "
                                   "forward pass of 2^22 rows",
                         "flops_per_ray": SUR_FLOPS_PER_RAY, "ms": fwd_ms}}


# ------------------------------------------------------------------ batched orbit
def orbit_section(args, ck, inputs, torch, flush):
    """The seeded 64-pose orbit (both cloaks and polarizations per pose, resolutions drawn from
    256^2 ... 3840x2160, 1 spp, DP5(4) tol 1e-9 FP64) in ONE batched render: one persistent integration
    kernel over every view, replayed as a CUDA graph.  The schedule (packet size, long-ray blocks, rays
    reserved per thread, cost-bucket resolution) comes from the autotuner, run on the same orbit with a
    quarter of each image side; the full orbit is timed with the default schedule and with the tuned one."""
    from paper_1209_6038_gb300 import autotune
    views = inputs.batched_views(64, 0)
    w = inputs.FULL
    c = ck.Cloak(ck.RADIAL).integrator(ck.DP45 if w.integrator == "dp45" else ck.RK4, w.h_or_tol, ck.FP64,
                                       w.max_steps)
    c.schedule(ck.SCHED_WAVEFRONT).stage_timing(True)
    small = [(v, p, eye, tgt, up, fov, torch.empty((max(1, H // 4), max(1, W // 4), 4), device="cuda"))
             for (v, p, eye, tgt, up, fov, W, H) in views]
    t0 = time.perf_counter()
    best, tune_ms = autotune.tune_schedule(c, lambda: ck.cloak_render_batch(c.h, small, 1, 0), key="orbit64/4",
                                           use_cache=False)
    tune_s = time.perf_counter() - t0
    del small
    outs = [(v, p, eye, tgt, up, fov, torch.empty((H, W, 4), device="cuda"))
            for (v, p, eye, tgt, up, fov, W, H) in views]
    rays = sum(o[-1].shape[0] * o[-1].shape[1] for o in outs)

    def timed_orbit(sched):
        autotune.apply(c, sched)
        ck.cloak_render_batch(c.h, outs, 1, 0)  # capture + first replay
        torch.cuda.synchronize()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ck.cloak_render_batch(c.h, outs, 1, 0)
        b.record()
        b.synchronize()
        return a.elapsed_time(b), c.stage_times()

    ms_default, _ = timed_orbit(autotune.DEFAULT_SCHEDULE)
    ms, st = timed_orbit(best)
    c.close()
    del outs
    return {"workload": "64 seeded orbit poses x 2 variants x 2 pols (256 views), resolutions from "
                        "{256x256, 1024x768, 1920x1080, 3840x2160}, 1 spp, DP45 tol=1e-9 FP64, one batched render",
            "views": len(views), "rays": rays, "value": rays / (ms / 1e3), "unit": "rays/s", "ms_per_step": ms,
            "warmup": 1, "steps": 1, "schedule": best, "default_schedule": autotune.DEFAULT_SCHEDULE,
            "ms_per_step_default_schedule": ms_default, "speedup_tuned_vs_default": ms_default / ms,
            "autotune": {"search": "coordinate search on the orbit at a quarter of each image side",
                         "seconds": tune_s, "ms": {str(k): v for k, v in tune_ms.items()}},
            "stage_ms": {"camera_entry_sort": st[0], "integrate": st[1], "exit_shade": st[2], "resolve": st[3]}}


def formulation_section(args, ck, torch):
    """Fermat form (Eq. 2 / Eq. 8, state (x, v)) against the Hamiltonian form (state (x, k)) on rays
    that a perfect cloak must pass undisturbed: in-plane extraordinary rays (direction across the axis,
    impact parameter b, height z) through both cloaks, whose exact exit is the vacuum line itself (exit
    point (sqrt(R2^2 - b^2), b, z), direction unchanged, optical time = the vacuum chord).  For each form
    and stepper setting (RK4 step h, DP5(4) tolerance) the section measures the largest relative error
    of exit point (/ R2), direction and time over all rays, and the time of one plain trace launch; then
    reports, per form, the cheapest setting that reaches 1e-8 (the paper's Sect. 4 comparison)."""
    n = 1 << 17
    R2 = 1.0
    g = torch.Generator(device="cpu").manual_seed(2024)
    b = (0.05 + 0.93 * torch.rand(n, generator=g, dtype=torch.float64)) * torch.where(
        torch.rand(n, generator=g) < 0.5, -1.0, 1.0).double()
    z = (torch.rand(n, generator=g, dtype=torch.float64) - 0.5) * 1.6
    rays = torch.zeros((n, 6), dtype=torch.float64)
    rays[:, 0], rays[:, 1], rays[:, 2], rays[:, 3] = -4.0, b, z, 1.0
    rays = rays.cuda()
    bx = b.cuda()
    ex = torch.stack([torch.sqrt(R2 * R2 - bx * bx), bx, z.cuda()], 1)
    tof_exact = 2 * torch.sqrt(R2 * R2 - bx * bx)
    out = torch.empty(n * ck.RECORD_BYTES, dtype=torch.uint8, device="cuda")
    settings = [(ck.RK4, 0.0125 / 2 ** k) for k in range(7)] + [(ck.DP45, 10.0 ** -e) for e in range(6, 14)]
    res = {}
    for form, fname in ((ck.FORM_FERMAT, "fermat"), (ck.FORM_HAMILTONIAN, "hamiltonian")):
        for variant, vname in ((ck.RADIAL, "radial"), (ck.AZIMUTHAL, "azimuthal")):
            c = ck.Cloak(variant, R2=R2)
            for kind, hv in settings:
                c.integrator(kind, hv, ck.FP64, 10_000_000).formulation(form)
                c.trace_rays(ck.POL_EXTRAORDINARY, rays, out)
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record()
                c.trace_rays(ck.POL_EXTRAORDINARY, rays, out)
                ev[1].record()
                ev[1].synchronize()
                f64 = out.view(torch.float64).view(n, 10)
                i32 = out.view(torch.int32).view(n, 20)
                ok = bool((i32[:, 17] == 1).all())
                err_pos = float((f64[:, 0:3] - ex).abs().max()) / R2
                err_dir = float((f64[:, 3:6] - rays[:, 3:6]).abs().max())
                err_tof = float(((f64[:, 6] - tof_exact).abs() / tof_exact).max())
                res[(fname, vname, kind, hv)] = {
                    "ms": ev[0].elapsed_time(ev[1]), "mean_steps": float(i32[:, 18].double().mean()),
                    "max_rel_err": max(err_pos, err_dir, err_tof) if ok else float("inf")}
            c.close()
    del out
    summary = {}
    for kind, kname in ((ck.RK4, "rk4"), (ck.DP45, "dp45")):
        for vname in ("radial", "azimuthal"):
            row = {}
            for fname in ("fermat", "hamiltonian"):
                hit = [(hv, r) for (f, v, k, hv), r in res.items()
                       if f == fname and v == vname and k == kind and r["max_rel_err"] <= 1e-8]
                if hit:
                    hv, r = min(hit, key=lambda t: t[1]["ms"])
                    row[fname] = {"h" if kind == ck.RK4 else "tol": hv, **r}
            if len(row) == 2:
                row["time_ratio_hamiltonian_over_fermat"] = row["hamiltonian"]["ms"] / row["fermat"]["ms"]
            summary[f"{kname}_{vname}"] = row
    return {"workload": f"{n} in-plane extraordinary rays per cloak (|b| in [0.05, 0.98] R2, |z| < 0.8), exact exit "
                        "= the vacuum line; plain trace launch; cheapest setting with max relative error <= 1e-8",
            "to_1e-8": summary,
            "sweep": [{"form": f, "variant": v, "stepper": "rk4" if k == ck.RK4 else "dp45", "h_or_tol": hv, **r}
                      for (f, v, k, hv), r in res.items()]}


# ------------------------------------------------------------------ native arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--ref-pixels", type=int, default=20000,
                    help="oracle pixels per image per step (enough rays per image to keep all host cores busy)")
    ap.add_argument("--cpu-pixels", type=int, default=100000, help="oracle pixels per image for cpu_baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-orbit", action="store_true")
    ap.add_argument("--no-formulation", action="store_true")
    ap.add_argument("--sur-epochs", type=int, default=60, help="stage-1 epochs of the surrogate's training")
    ap.add_argument("--profile-image", default=None,
                    help="VARIANT,MODE,ELEV: render only this image twice (for profilers), e.g. 1,1,20")
    ap.add_argument("--sur-fp16", action="store_true",
                    help="with --profile-gemm: the network's FP16 inference (cloak_surrogate_set_precision)")
    ap.add_argument("--profile-gemm", action="store_true",
                    help="run the surrogate network's forward pass (seeded initial weights) twice on 2^20 rows, "
                         "for profilers")
    ap.add_argument("--profile-batch", action="store_true",
                    help="render the step's 12 images through the batched path twice at --width x --height "
                         "(default 480x270), for profilers")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed_df"],
                    help="arithmetic of --profile-batch: FP64, or FP32 stepping with the band near R1 in FP64 "
                         "(mixed) or in double-float (mixed_df)")
    ap.add_argument("--width", type=int, default=None)
    ap.add_argument("--height", type=int, default=None)
    ap.add_argument("--schedule", default="batched", choices=["plain", "wavefront", "batched"])
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1209_6038_gb300 import build as pbuild
    if rank == 0:
        pbuild.build()
    if ws > 1:
        dist.barrier()
    from paper_1209_6038_gb300 import cloak as ck
    from paper_1209_6038_gb300 import inputs, replicas
    ck.load()
    w = inputs.FULL
    stream = torch.cuda.current_stream()
    if args.profile_image:
        v, m, e = args.profile_image.split(",")
        W, H = args.width or w.width, args.height or w.height
        eye, tgt, up = inputs.camera_pose(float(e))
        c = ck.Cloak(int(v)).camera(eye, tgt, up, w.hfov_deg, W, H)
        c.integrator(ck.DP45 if w.integrator == "dp45" else ck.RK4, w.h_or_tol, ck.FP64, w.max_steps)
        c.schedule(ck.SCHED_PLAIN if args.schedule == "plain" else ck.SCHED_WAVEFRONT)
        img = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        for _ in range(2):
            c.render(int(m), w.spp, w.seed, out=img)
        torch.cuda.synchronize()
        print(json.dumps({"profile_image": args.profile_image, "width": W, "height": H,
                          "mean_rgba": img.mean(dim=(0, 1)).tolist()}))
        c.close()
        return 0

    if args.profile_gemm:
        c = ck.Cloak(ck.RADIAL)
        ck.cloak_surrogate_params(c.h, ck.cloak_surrogate_params(c.h))  # creates the network (seeded weights)
        ck.cloak_surrogate_set_precision(c.h, args.sur_fp16)
        n = 1 << 20
        g = torch.Generator(device="cuda").manual_seed(0)
        x = torch.rand((n, 7), device="cuda", generator=g) * 2 - 1
        y = torch.empty((n, 5), device="cuda")
        for _ in range(2):
            ck.cloak_surrogate_forward(c.h, x, y)
        torch.cuda.synchronize()
        print(json.dumps({"profile_gemm": True, "fp16": args.sur_fp16, "rows": n, "mean_out": y.mean(0).tolist()}))
        c.close()
        return 0
    if args.profile_batch:
        W, H = args.width or 480, args.height or 270
        prec = {"fp64": ck.FP64, "mixed": ck.MIXED, "mixed_df": ck.MIXED_FF}[args.precision]
        c = ck.Cloak(ck.RADIAL).integrator(ck.DP45 if w.integrator == "dp45" else ck.RK4, w.h_or_tol, prec,
                                           w.max_steps)
        c.schedule(ck.SCHED_WAVEFRONT)
        views = []
        for v, m, e in w.images:
            eye, tgt, up = inputs.camera_pose(e)
            views.append((v, m, eye, tgt, up, w.hfov_deg,
                          torch.empty((H, W, 4), dtype=torch.float32, device="cuda")))
        for _ in range(2):
            ck.cloak_render_batch(c.h, views, w.spp, w.seed)
        torch.cuda.synchronize()
        print(json.dumps({"profile_batch": True, "precision": args.precision, "width": W, "height": H,
                          "images": len(views),
                          "mean_rgba": torch.stack([v[-1].mean(dim=(0, 1)) for v in views]).mean(0).tolist()}))
        c.close()
        return 0

    def make_handles(schedule, precision=None):
        hs = {}
        for v in w.variants:
            for e in w.elevations:
                eye, tgt, up = inputs.camera_pose(e)
                c = ck.Cloak(v).camera(eye, tgt, up, w.hfov_deg, w.width, w.height)
                c.integrator(ck.DP45 if w.integrator == "dp45" else ck.RK4, w.h_or_tol,
                             ck.FP64 if precision is None else precision, w.max_steps)
                c.schedule(schedule)
                hs[(v, e)] = c
        return hs

    imgs = [torch.empty((w.height, w.width, 4), dtype=torch.float32, device="cuda") for _ in w.images]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    integ_kind = ck.DP45 if w.integrator == "dp45" else ck.RK4

    class PerImage:
        """one handle per (variant, elevation), one render call per image"""

        def __init__(self, schedule, precision=ck.FP64):
            self.hs = make_handles(schedule, precision)
            for c in self.hs.values():
                c.stage_timing(True)
            # kernels per image: entry, sort scan, sort scatter, integrate, exit, resolve (wavefront); one (plain)
            self.launches = (6 if schedule == ck.SCHED_WAVEFRONT else 1) * len(w.images)

        def step(self, stage_ms=None):
            for i, (v, m, e) in enumerate(w.images):
                c = self.hs[(v, e)]
                c.render(m, w.spp, w.seed, out=imgs[i])
                if stage_ms is not None:
                    for k, t in enumerate(c.stage_times()):
                        stage_ms[k] += t

        def close(self):
            for c in self.hs.values():
                c.close()

    class Batched:
        """all images of the step in one cloak_render_batch call (one persistent integration kernel,
        replayed CUDA graph)"""

        def __init__(self, precision=ck.FP64, images=None):
            self.h = ck.Cloak(ck.RADIAL).integrator(integ_kind, w.h_or_tol, precision, w.max_steps)
            self.h.schedule(ck.SCHED_WAVEFRONT).stage_timing(True)
            self.views = []
            for i, (v, m, e) in enumerate(w.images):
                eye, tgt, up = inputs.camera_pose(e)
                self.views.append((v, m, eye, tgt, up, w.hfov_deg, (images or imgs)[i]))
            # kernels per step: entry, sort scan, sort scatter, integrate, exit, resolve (the view-table copy
            # and the queue-header memset of the same graph are not kernels)
            self.launches = 6

        def step(self, stage_ms=None):
            ck.cloak_render_batch(self.h.h, self.views, w.spp, w.seed)
            if stage_ms is not None:
                for k, t in enumerate(self.h.stage_times()):
                    stage_ms[k] += t

        def close(self):
            self.h.close()

    def timed(runner, warmup, steps, sampler=None, collective=True):
        """mean ms per step (the slowest rank's when collective), per-step ms, mean stage ms; sections that
        run on rank 0 alone pass collective=False"""
        coll = collective and ws > 1
        for _ in range(warmup):
            runner.step()
        torch.cuda.synchronize()
        if coll:
            dist.barrier()
        torch.cuda.synchronize()
        stage_ms = [0.0, 0.0, 0.0, 0.0]
        ms = []
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            for _ in range(steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                runner.step(stage_ms)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
        torch.cuda.synchronize()
        if coll:
            dist.barrier()
        tot = replicas.max_over_ranks(sum(ms), device="cuda") if coll else sum(ms)  # the slowest rank's time
        return tot / steps, ms, [x / steps for x in stage_ms]

    if args.schedule == "batched":
        main_runner = Batched()
    else:
        main_runner = PerImage(ck.SCHED_WAVEFRONT if args.schedule == "wavefront" else ck.SCHED_PLAIN)
    sampler = ClockSampler(local)
    ms_step, ms_list, stages = timed(main_runner, args.warmup, args.steps, sampler)
    rays_step = w.rays
    value = replicas.whole_job_rate(rays_step, ms_step / 1e3, ws)
    clocks = sampler.summary()

    from paper_1209_6038_gb300 import alu_peaks
    live = alu_peaks.measure(seconds=1.0, repeats=1)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(w),
           "schedule": args.schedule, "clocks": clocks,
           "gpu_launches": main_runner.launches * args.steps,
           "alu_peaks_tflops": {"fp64": FP64_PEAK_TFLOPS, "fp32": FP32_PEAK_TFLOPS, "source": ALU_PEAK_SOURCE,
                                "fp64_this_run": live["fp64"]["tflops"], "fp32_this_run": live["fp32"]["tflops"]},
           "stage_ms_per_step": {"camera_entry_sort": stages[0], "integrate": stages[1], "exit_shade": stages[2],
                                 "resolve": stages[3]}}

    # ---- end to end through the public API: render and copy every image to pinned host memory (measured
    # right after the device-timed steps, on the same handle and views)
    if not args.no_e2e:
        # Steps run back to back, each rendering all views and copying its images to pinned host memory.
        # Batched schedule: two output sets (two handles), so that the copy of step k (on a copy stream)
        # overlaps the render of step k + 1 -- a render waits only for the copy that last read its set.
        sets = [(main_runner, imgs)]
        if args.schedule == "batched":
            imgs2 = [torch.empty_like(im) for im in imgs]
            sets.append((Batched(images=imgs2), imgs2))
        host = [[torch.empty_like(im, device="cpu").pin_memory() for im in ims] for _, ims in sets]
        for r, _ in sets:
            r.step()
        torch.cuda.synchronize()
        cs = torch.cuda.Stream()
        copied = [None] * len(sets)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            j = k % len(sets)
            r, ims = sets[j]
            if copied[j] is not None:
                torch.cuda.current_stream().wait_event(copied[j])
            flush.zero_()  # L2 flushed between steps, as for the device-timed steps
            r.step()
            rendered = torch.cuda.Event()
            rendered.record()
            with torch.cuda.stream(cs):
                cs.wait_event(rendered)
                for hb, im in zip(host[j], ims):
                    hb.copy_(im, non_blocking=True)
                copied[j] = torch.cuda.Event()
                copied[j].record(cs)
        torch.cuda.synchronize()
        e2e_total = time.perf_counter() - t0
        e2e_s = replicas.max_over_ranks(e2e_total / args.steps, device="cuda")  # the slowest rank's
        e2e = replicas.whole_job_rate(rays_step, e2e_s, ws)
        out["e2e"] = {"value": e2e, "unit": UNIT, "ms_per_step": 1e3 * e2e_total / args.steps,
                      "h2d_bytes_per_step": VIEW_TABLE_BYTES * len(w.images) if args.schedule == "batched" else 0,
                      "d2h_bytes_per_step": sum(im.numel() * 4 for im in imgs),
                      "note": "host wall time of steps run back to back; inputs are camera and integrator parameters "
                              "(host structs passed through the C ABI; the batched render copies its view table to "
                              "the device each step); outputs are the 12 float4 images copied to pinned host memory "
                              "every step, the copy of step k overlapping the render of step k + 1 (two output sets)"}
        if len(sets) > 1:
            sets[1][0].close()
            del imgs2


    if rank == 0:
        # ---- records pass (untimed): step counts for the roofline, sampled rays for the error
        rec_handles = make_handles(ck.SCHED_WAVEFRONT)
        rec_buf = torch.empty(w.rays_per_image * ck.RECORD_BYTES, dtype=torch.uint8, device="cuda")
        flops = 0.0
        steps_total = 0
        status_hist = np.zeros(8, np.int64)
        gpu_samples = []
        for idx, (v, m, e) in enumerate(w.images):
            rec_handles[(v, e)].render_records(m, w.spp, w.seed, out=rec_buf)
            i32 = rec_buf.view(torch.int32).view(-1, 20)   # cloak_record: tile_id, status, steps at 16, 17, 18
            status = i32[:, 17].long()
            steps_img = int(i32[:, 18].long().sum().item())
            steps_total += steps_img
            flops += steps_img * flops_per_step(v, m, 1 if w.integrator == "dp45" else 0)
            status_hist += torch.bincount(status, minlength=8).cpu().numpy()[:8]
            pix = sample_pixels(w, idx, args.cpu_pixels)
            sel = torch.from_numpy((pix[:, None] * w.spp + np.arange(w.spp)[None, :]).reshape(-1)).cuda()
            gpu_samples.append(ck.records_to_numpy(rec_buf.view(-1, ck.RECORD_BYTES)[sel].reshape(-1)))
        del rec_buf
        kname = {"batched": "k_wf_integrate<any medium> (1 launch per step, all 12 images)",
                 "wavefront": "k_wf_integrate (12 launches per step)",
                 "plain": "k_render_plain (12 launches per step)"}[args.schedule]
        achieved = flops / (stages[1] / 1e3) / 1e12
        out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": achieved / FP64_PEAK_TFLOPS,
                           "traffic": INTEGRATE_TRAFFIC_BYTES if args.schedule == "batched" else None,
                           "traffic_note": "ncu dram bytes of a 480x270 x 4 spp capture of the same views, scaled by "
                                           "samples" if args.schedule == "batched" else None,
                           "peak_source": ALU_PEAK_SOURCE + " (FP64)", "kernel": kname,
                           "kernel_ms_per_step": stages[1]}
        # camera rays integrated through the cloak: exited, exited after the metal mirror, TIR at the exit,
        # step limit, singular (not: missed, no transmitted mode at entry, metal cap disc hit from outside)
        in_cloak = int(status_hist[[1, 2, 4, 5, 6]].sum())
        out["work"] = {"integrator_steps_per_step": steps_total, "fp64_flops_per_step": flops,
                       "status_hist": {ck.RAY_STATUS[i]: int(status_hist[i]) for i in range(8)},
                       "in_cloak_rays_per_step": in_cloak,
                       "in_cloak_rays_per_s": in_cloak / (ms_step / 1e3),
                       "rk_step_attempts_per_s": steps_total / (ms_step / 1e3)}

        # ---- CPU oracle on a bounded sample, and the exit-direction error against it
        cores = os.cpu_count() or 1
        nr, dt, orecs = run_oracle_sample(w, args.cpu_pixels, cores)
        # one core on a sample a twelfth the size (seeded the same way): the per-core rate
        nr1, dt1, _ = run_oracle_sample(w, max(1, args.cpu_pixels // 12), 1)
        # the small workload (radial e, 128x96 x 1 spp, RK4 h = 1e-3) in full, all cores
        ws_small = inputs.SMALL
        nrs, dts, _ = run_oracle_sample(ws_small, ws_small.width * ws_small.height, cores)
        g = np.concatenate(gpu_samples)
        o = np.concatenate(orecs)
        ref, lim64, und = reference_records(w, o, args.cpu_pixels)
        fin = np.isin(ref["status"], [0, 1, 2, 7]) & (g["status"] == ref["status"])
        err = angles(g["exit_dir"][fin], ref["exit_dir"][fin])
        px_g = (g["tile_id"] != ref["tile_id"]) | (g["status"] != ref["status"])
        px_diff = px_g.reshape(-1, w.spp).any(1)
        out["cpu_baseline"] = {"value": nr / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{args.cpu_pixels} seeded pixels x {w.spp} spp from each of the "
                                         f"{len(w.images)} images ({nr} rays), {dt:.1f} s",
                               "single_core": {"value": nr1 / dt1, "unit": UNIT, "cores": 1,
                                               "sample": f"{max(1, args.cpu_pixels // 12)} seeded pixels x {w.spp} spp "
                                                         f"per image ({nr1} rays), {dt1:.1f} s"},
                               "small_workload_full": {"value": nrs / dts, "unit": UNIT, "cores": cores,
                                                       "sample": f"{ws_small.name}, every pixel ({nrs} rays), "
                                                                 f"{dts:.2f} s"}}
        e_det = err[~und[fin]]
        e_und = err[und[fin]]
        out["accuracy_vs_oracle"] = {
            "reference": "FP64 oracle; binary128 oracle (same source, tol 1e-9) on the rays the FP64 oracle does not "
                         "determine (tests/golden/fp64_undetermined_rays.txt)",
            "max_exit_dir_err_rad": float(err.max(initial=0)),
            "max_exit_dir_err_rad_fp64_oracle_determined": float(e_det.max(initial=0)),
            "max_exit_dir_err_rad_vs_binary128": float(e_und.max(initial=0)),
            "rays_vs_binary128": int(und.sum()),
            "rays_over_1e-9_rad": int((err > 1e-9).sum()),
            "rays_over_bar": int((err > lim64[fin]).sum()),
            "rays_with_widened_bar": int((lim64 > 1e-9).sum()),
            "p999_exit_dir_err_rad": float(np.quantile(err, 0.999)) if len(err) else 0.0,
            "rays_compared": int(fin.sum()),
            "status_mismatch": int((g["status"] != ref["status"]).sum()),
            "status_mismatch_vs_fp64_oracle_alone": int((g["status"] != o["status"]).sum()),
            "max_exit_dir_err_rad_vs_fp64_oracle_alone": float(
                angles(g["exit_dir"][fin & (g["status"] == o["status"])], o["exit_dir"][fin & (g["status"] == o["status"])]).max(initial=0)),
            "pixels_tile_or_status_differs_frac": float(px_diff.mean())}

        # ---- the precision form: the same workload with FP32 stepping (mixed), against the oracle sample; the
        # band near R1 in FP64 ("mixed") and in double-float ("mixed_df_band")
        for prec, key, band in ((ck.MIXED, "mixed", "f64 band r < R1 + 0.02"),
                                (ck.MIXED_FF, "mixed_df_band", "double-float (FP32 pair) band r < R1 + 0.02")):
            if args.no_mixed:
                break
            mixed_runner = Batched(prec) if args.schedule == "batched" else PerImage(ck.SCHED_WAVEFRONT, prec)
            sched, tune_ms, tune_s = None, None, 0.0
            if args.schedule == "batched":
                # the step schedule from the autotuner, on this step itself (coordinate search, one timed
                # render per candidate)
                from paper_1209_6038_gb300 import autotune
                t0 = time.perf_counter()
                # two timed renders per candidate (the faster counts): one-render timings differ by ~3 % from
                # call to call, as much as the knobs' effects near the optimum
                sched, tune_ms = autotune.tune_schedule(mixed_runner.h, mixed_runner.step, key=f"full12|{key}",
                                                        reps=2, use_cache=False, start=autotune.MIXED_SCHEDULE)
                tune_s = time.perf_counter() - t0
            mms, _, mstages = timed(mixed_runner, 1, 2, collective=False)
            mixed_runner.close()
            mh = make_handles(ck.SCHED_WAVEFRONT, precision=prec)
            rec_buf = torch.empty(w.rays_per_image * ck.RECORD_BYTES, dtype=torch.uint8, device="cuda")
            msamples = []
            mflops = 0.0
            for idx, (v, m, e) in enumerate(w.images):
                mh[(v, e)].render_records(m, w.spp, w.seed, out=rec_buf)
                msteps = int(rec_buf.view(torch.int32).view(-1, 20)[:, 18].long().sum().item())
                mflops += msteps * flops_per_step(v, m, 1 if w.integrator == "dp45" else 0)
                pix = sample_pixels(w, idx, args.cpu_pixels)
                sel = torch.from_numpy((pix[:, None] * w.spp + np.arange(w.spp)[None, :]).reshape(-1)).cuda()
                msamples.append(ck.records_to_numpy(rec_buf.view(-1, ck.RECORD_BYTES)[sel].reshape(-1)))
            del rec_buf
            for c in mh.values():
                c.close()
            gm = np.concatenate(msamples)
            lim32, flip32 = fp32_bars(w, args.cpu_pixels)
            fin = np.isin(ref["status"], [0, 1, 2, 7]) & (gm["status"] == ref["status"])
            errm = angles(gm["exit_dir"][fin], ref["exit_dir"][fin])
            det32 = lim32[fin] <= 1e-5
            pxm = ((gm["tile_id"] != ref["tile_id"]) | (gm["status"] != ref["status"])).reshape(-1, w.spp).any(1)
            out[key] = {"value": ws * rays_step / (mms / 1e3), "unit": UNIT, "ms_per_step": mms, "warmup": 1,
                        "steps": 2, "schedule": args.schedule,
                        "dtype": "f32 stepping, float-float state, " + band,
                        "integrate_ms_per_step": mstages[1], "speedup_vs_fp64": ms_step / mms,
                        "schedule": sched,
                        "autotune": None if sched is None else {
                            "seconds": tune_s, "default_ms": tune_ms["default"],
                            "ms": {k: v for k, v in tune_ms.items()},
                            "search": "coordinate search over packet, long-ray blocks, cost scale and rays "
                                      "reserved per thread, the faster of two timed batched steps per candidate"},
                        "roofline": {"bound": "alu", "achieved": mflops / (mstages[1] / 1e3) / 1e12,
                                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                     "frac": mflops / (mstages[1] / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
                                     "peak_source": ALU_PEAK_SOURCE + " (FP32)",
                                     "note": "algorithmic flops of the step attempts (the FP64 path's per-attempt "
                                             "count, band steps included) over the integration kernel's time; the "
                                             "kernel is bound by latency and lane divergence, not an FP32 pipe "
                                             "(ncu summary of k_wf_integrate, mixed, 480x270 x 4 spp)"},
                        "accuracy_vs_oracle": {
                            "max_exit_dir_err_rad": float(errm.max(initial=0)),
                            "max_exit_dir_err_rad_fp32_determined": float(errm[det32].max(initial=0)),
                            "rays_fp32_determined_over_1e-5": int((errm[det32] > 1e-5).sum()),
                            "rays_with_widened_bar": int((~det32).sum()),
                            "rays_over_bar": int((errm > lim32[fin]).sum()),
                            "p999_exit_dir_err_rad": float(np.quantile(errm, 0.999)),
                            "rays_over_1e-5_rad": int((errm > 1e-5).sum()),
                            "rays_compared": int(fin.sum()),
                            "status_changes": int((gm["status"] != ref["status"]).sum()),
                            "status_changes_fp32_determined": int(((gm["status"] != ref["status"]) & ~flip32).sum()),
                            "pixels_tile_or_status_differs_frac": float(pxm.mean()),
                            "bar": "min(1e-4, max(1e-5, 100 D32)), D32 the distance an FP32 model of the oracle moves the "
                                   "ray (tests/golden/fp32_sensitive_rays.txt)"}}
        for c in rec_handles.values():
            c.close()

        # ---- the learned surrogate with integrator fallback (3840x2160, 1 spp, the same views)
        if not args.no_surrogate:
            out["surrogate"] = surrogate_section(args, ck, inputs, torch, np, flush)

        # ---- the batched form: 64-pose orbit, 256 views, one persistent launch
        if not args.no_orbit:
            out["batched_orbit"] = orbit_section(args, ck, inputs, torch, flush)

        # ---- Fermat against Hamiltonian ray equations, time to 1e-8 on perfect-cloaking rays
        if not args.no_formulation:
            out["formulation"] = formulation_section(args, ck, torch)

    # ---- comparators on the same workload: per-image wavefront and the plain FP64 integrator
    if not args.no_plain:
        for name, sched in (("per_image_wavefront_fp64", ck.SCHED_WAVEFRONT), ("plain_fp64", ck.SCHED_PLAIN)):
            if (args.schedule == "wavefront" and sched == ck.SCHED_WAVEFRONT) or \
                    (args.schedule == "plain" and sched == ck.SCHED_PLAIN):
                continue
            r = PerImage(sched)
            pms, _, _ = timed(r, 1, 1)
            r.close()
            out[name] = {"value": ws * rays_step / (pms / 1e3), "unit": UNIT, "ms_per_step": pms, "warmup": 1,
                         "steps": 1}
        if "plain_fp64" in out:
            out["speedup_vs_plain_fp64"] = out["plain_fp64"]["ms_per_step"] / ms_step

    main_runner.close()
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


if __name__ == "__main__":
    sys.exit(main())
