"""Writes fp32_sensitive_rays.txt: the sampled rays of the 1920x1080 workload (the sample of
make_undetermined_rays.py) that FP32 arithmetic cannot determine to the mixed-precision bar of 1e-5 rad.
Calls only oracle/ (and the seeded input layout of the package's inputs module).

Every sampled ray is traced by the oracle in long double twice: exactly, and as a model of the mixed path's
FP32 arithmetic (right-hand sides of Eq. 2 / Eq. 8 and stage velocities rounded to FP32 outside the band
r < R1 + 0.02, FP64 stage points inside it).  D32 is the exit-direction distance between the two runs; the
file lists the rays with D32 > 1e-7 rad (100 D32 above the 1e-5 bar), or whose status the model changes.

  python tests/golden/make_fp32_sensitive_rays.py [--pixels 100000]
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fp32_sensitive_rays.txt")
SAMPLE_SEED = 12345
LISTED = 1e-7  # 100 x D32 above the 1e-5 bar: the rays whose bar widens


def _angle(a, b):
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cr, np.sum(a * b, axis=-1))


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--pixels", type=int, default=100000)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args(argv)
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle as O
    from oracle import build as obuild
    from paper_1209_6038_gb300 import inputs
    for k in ("ld", "ld_f32"):
        obuild.build_ext(k)
    w = inputs.FULL
    t0 = time.time()
    lines = []
    for idx, (v, m, e) in enumerate(w.images):
        eye, tgt, up = inputs.camera_pose(e)
        cam = O.Camera(eye, tgt, up, w.hfov_deg, w.width, w.height)
        pix = inputs.sample_pixels(w, idx, args.pixels, SAMPLE_SEED)
        integ = O.Integrator(O.DP45, w.h_or_tol, w.max_steps)
        _, rld = O.render(O.Cloak(v), integ, cam, m, w.spp, w.seed, pixels=pix, precision="ld")
        _, rf = O.render(O.Cloak(v), integ, cam, m, w.spp, w.seed, pixels=pix, precision="ld_f32")
        fin = np.isin(rld["status"], [0, 1, 2, 7])
        d32 = np.where(fin, _angle(rld["exit_dir"], rf["exit_dir"]), 0.0)
        flip = rld["status"] != rf["status"]
        sel = np.nonzero((d32 > LISTED) | flip)[0]
        samp = (pix[:, None] * w.spp + np.arange(w.spp)[None, :]).reshape(-1)
        lines += [f"{idx} {int(samp[k])} {d32[k]:.3e} {int(flip[k])}" for k in sel]
        print(f"image {idx}: {len(sel)} listed ({time.time() - t0:.0f} s)", flush=True)
    with open(args.out, "w") as f:
        f.write("# Rays of the 1920x1080 x 4 spp workload (both cloaks, Eqs. 14 / 15; both polarisations;\n"
                "# elevations 0/20/45 deg; DP5(4) at 1e-9) that a model of FP32 arithmetic moves by more than\n"
                f"# {LISTED:g} rad, or whose status it changes, out of {args.pixels} seeded pixels per image\n"
                f"# (inputs.sample_pixels, seed {SAMPLE_SEED}).  Model: the oracle in long double with its right-hand\n"
                "# sides and stage velocities rounded to FP32 outside r < R1 + 0.02, against the exact long-double\n"
                "# run.  Written by tests/golden/make_fp32_sensitive_rays.py (oracle only).\n"
                "# Columns: image index, flat sample index (pixel * spp + sample), D32 (rad), status changed (0/1).\n")
        for ln in lines:
            f.write(ln + "\n")
    print(f"wrote {len(lines)} rays ({time.time() - t0:.0f} s)")
    return 0


if __name__ == "__main__":
    sys.exit(main())
