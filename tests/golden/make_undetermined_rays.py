"""Writes fp64_undetermined_rays.txt: the reference for the sampled rays of the 1920x1080 workload whose
integration (Sect. 2, Eq. 2 / Eq. 8, Dormand-Prince 5(4) at tolerance 1e-9) the FP64 oracle does not
determine to 1e-10.  Calls only oracle/ (and the seeded input layout of the package's inputs module).

For every image of the workload (both cloaks of Eqs. 14 / 15, both polarisations, elevations 0/20/45 deg,
4 jittered samples per pixel) and the seeded pixel sample the tests and the benchmark check:
  1. the oracle traces every sampled ray in FP64 and, from the same source, in long double;
  2. a ray is "undetermined" when the two disagree -- status, or exit direction / exit point / time of
     flight / weight by more than 1e-10: FP64 rounding changes the oracle's result there.  Near r = R1 this is the
     literal Cartesian form of Eq. 8 losing digits to cancellation (its right-hand side is off by ~1e-3
     relative at r - R1 = 1e-5 in FP64), which also inflates its step counts by up to 80x;
  3. for those rays the same oracle source runs in IEEE binary128 (_Float128): at tolerance 1e-9 -- the
     reference the GPU's FP64 path is held to -- at 1e-12 -- the converged limit, for the truncation
     error of the method -- and at 1e-9 with every state and stage point rounded to FP64 (D64 = its
     distances from the exact run, per field: how far FP64 states alone move the ray, the best an FP64
     integrator can determine).

  python tests/golden/make_undetermined_rays.py [--pixels 100000] [--procs 8]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fp64_undetermined_rays.txt")
SAMPLE_SEED = 12345
THRESH = 1e-10


def _angle(a, b):
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cr, np.sum(a * b, axis=-1))


def _camera(O, inputs, w, e):
    eye, tgt, up = inputs.camera_pose(e)
    return O.Camera(eye, tgt, up, w.hfov_deg, w.width, w.height)


def _quad_job(args):
    """One ray (image, flat sample index): binary128 at 1e-9, at 1e-12, and at 1e-9 with FP64 states."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as O
    from paper_1209_6038_gb300 import inputs
    w = inputs.FULL
    idx, samp = args
    v, m, e = w.images[idx]
    cam = _camera(O, inputs, w, e)
    pix, s = np.array([samp // w.spp]), samp % w.spp
    out = []
    for prec, tol in (("q", 1e-9), ("q", 1e-12), ("q_s64", 1e-9)):
        _, r = O.render(O.Cloak(v), O.Integrator(O.DP45, tol, 100_000_000), cam, m, w.spp, w.seed, pixels=pix,
                        nthreads=1, precision=prec)
        out.append(r[s])
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--pixels", type=int, default=100000, help="sampled pixels per image")
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args(argv)
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as O
    from oracle import build as obuild
    from paper_1209_6038_gb300 import inputs
    for k in ("ld", "q", "q_s64"):
        obuild.build_ext(k)
    w = inputs.FULL
    t0 = time.time()
    rows = []
    for idx, (v, m, e) in enumerate(w.images):
        cam = _camera(O, inputs, w, e)
        pix = inputs.sample_pixels(w, idx, args.pixels, SAMPLE_SEED)
        integ = O.Integrator(O.DP45, w.h_or_tol, w.max_steps)
        _, r64 = O.render(O.Cloak(v), integ, cam, m, w.spp, w.seed, pixels=pix)
        _, rld = O.render(O.Cloak(v), integ, cam, m, w.spp, w.seed, pixels=pix, precision="ld")
        und = ((r64["status"] != rld["status"]) | (_angle(r64["exit_dir"], rld["exit_dir"]) > THRESH) |
               (np.linalg.norm(r64["exit_pos"] - rld["exit_pos"], axis=-1) > THRESH) |
               (np.abs(r64["tof"] - rld["tof"]) > THRESH) | (np.abs(r64["weight"] - rld["weight"]) > THRESH))
        samp = (pix[:, None] * w.spp + np.arange(w.spp)[None, :]).reshape(-1)
        rows += [(idx, int(s)) for s in samp[und]]
        print(f"image {idx}: {int(und.sum())} undetermined of {len(samp)} ({time.time() - t0:.0f} s)", flush=True)
    with mp.get_context("spawn").Pool(args.procs) as pool:
        res = pool.map(_quad_job, rows, chunksize=1)
    print(f"binary128 runs done ({time.time() - t0:.0f} s)", flush=True)
    with open(args.out, "w") as f:
        f.write("# Reference for the rays of the 1920x1080 x 4 spp workload (both cloaks, Eqs. 14 / 15; both\n"
                "# polarisations; elevations 0/20/45 deg; DP5(4) at tolerance 1e-9 on Eq. 2 / Eq. 8, Sect. 2 and 4)\n"
                f"# whose FP64 oracle result differs from the same oracle in long double by more than {THRESH:g}\n"
                f"# (status, exit direction, exit point, time of flight or weight), out of {args.pixels} seeded pixels per\n"
                f"# image (inputs.sample_pixels, seed {SAMPLE_SEED}).  Written by tests/golden/"
                "make_undetermined_rays.py (oracle only).\n"
                "# Columns: image index, flat sample index (pixel * spp + sample); then the oracle in binary128 at\n"
                "# tolerance 1e-9: status, step attempts, exit direction (3), exit point (3), time of flight, weight,\n"
                "# tile id; the exit direction (3) at tolerance 1e-12 (the converged limit); D64 of the exit direction\n"
                "# (rad), exit point, time of flight and weight: their change between the binary128 run at 1e-9 and\n"
                "# the same run with FP64 states.\n")
        for (idx, samp), (q9, q12, qs) in zip(rows, res):
            vals = [idx, samp, int(q9["status"]), int(q9["steps"])]
            vals += [f"{x:.17g}" for x in q9["exit_dir"]] + [f"{x:.17g}" for x in q9["exit_pos"]]
            vals += [f"{q9['tof']:.17g}", f"{q9['weight']:.17g}", int(q9["tile_id"])]
            vals += [f"{x:.17g}" for x in q12["exit_dir"]]
            vals += [f"{float(_angle(q9['exit_dir'], qs['exit_dir'])):.3e}",
                     f"{float(np.abs(q9['exit_pos'] - qs['exit_pos']).max()):.3e}",
                     f"{abs(float(q9['tof'] - qs['tof'])):.3e}", f"{abs(float(q9['weight'] - qs['weight'])):.3e}"]
            f.write(" ".join(str(x) for x in vals) + "\n")
    print(f"wrote {len(rows)} rays to {args.out} ({time.time() - t0:.0f} s)")
    return 0


if __name__ == "__main__":
    sys.exit(main())
