"""Writes tests/golden/parity/<case>.txt: for every GPU parity case of tests/parity_cases.py, the rays whose
result the FP64 oracle does not determine, with their reference from the same oracle source in IEEE
binary128.  Calls only oracle/ (and the seeded inputs of tests/parity_cases.py).

A ray is undetermined when the oracle in FP64 and in long double disagree: status, or exit direction (rad),
exit point, time of flight or weight by more than 1e-10 (FP64 rounding moves the oracle's result there;
near r = R1 the literal Cartesian form of Eq. 8 loses digits to cancellation).  For those rays the file
holds the binary128 result at the case's own step or tolerance (status, step attempts, exit direction,
exit point, time of flight, weight, tile) and D64 per field (exit direction, exit point, time of flight,
weight): the distance between that run and the same run with every state and stage point rounded to
FP64, how far FP64 states alone move the ray.

For the cases of the mixed-precision path it also writes <case>.f32.txt: the rays that a model of FP32
arithmetic (long double with FP32 right-hand sides and stage velocities outside the band r < R1 + 0.02)
moves by D32 > 1e-7 rad (100 D32 above the 1e-5 bar), or whose status it changes.

  python tests/golden/make_parity_references.py [--procs 8] [--only NAME ...]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT_DIR = os.path.join(HERE, "parity")
THRESH = 1e-10
F32_LISTED = 1e-7  # D32 above which the 1e-5 bar widens (100 x D32 > 1e-5): listed


def _setup():
    for p in (ROOT, os.path.join(ROOT, "tests")):
        if p not in sys.path:
            sys.path.insert(0, p)


def angles(a, b):
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    return np.arctan2(cr, np.sum(a * b, axis=-1))


def undetermined(r64, rld):
    return ((r64["status"] != rld["status"]) | (angles(r64["exit_dir"], rld["exit_dir"]) > THRESH) |
            (np.abs(r64["exit_pos"] - rld["exit_pos"]).max(1) > THRESH) | (np.abs(r64["tof"] - rld["tof"]) > THRESH) |
            (np.abs(r64["weight"] - rld["weight"]) > THRESH))


def _one(args):
    """binary128 (exact and with FP64 states) for ray `k` of case `name`."""
    _setup()
    import oracle as O
    import parity_cases as P
    name, k = args
    s = P.materialise(P.cases()[name])
    if s["kind"] == "rays":
        sub = dict(s, rays=s["rays"][k:k + 1])
        pick = 0
    else:
        spp = s["spp"]
        pix = s["pixels"] if s["pixels"] is not None else np.arange(s["width"] * s["height"])
        sub = dict(s, pixels=np.array([pix[k // spp]]))
        pick = k % spp
    q = P.oracle_records(O, sub, precision="q", nthreads=1)[pick]
    qs = P.oracle_records(O, sub, precision="q_s64", nthreads=1)[pick]
    return q, qs


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", nargs="*", default=None)
    args = ap.parse_args(argv)
    _setup()
    import oracle as O
    from oracle import build as obuild
    import parity_cases as P
    for k in ("ld", "q", "q_s64", "ld_f32"):
        obuild.build_ext(k)
    os.makedirs(OUT_DIR, exist_ok=True)
    allc = P.cases()
    names = args.only or sorted(allc)
    t0 = time.time()
    jobs, per_case = [], {}
    for name in names:
        s = allc[name]
        r64 = P.oracle_records(O, s)
        rld = P.oracle_records(O, s, precision="ld")
        idx = np.nonzero(undetermined(r64, rld))[0]
        per_case[name] = (len(r64), idx)
        jobs += [(name, int(k)) for k in idx]
        print(f"{name}: {len(idx)} undetermined of {len(r64)} ({time.time() - t0:.0f} s)", flush=True)
    # FP32 model of the mixed path's cases: D32 of every ray (long double, FP32 right-hand sides and stage
    # velocities outside the band r < R1 + 0.02, against the exact long-double run)
    f32 = {}
    for name in names:
        if not allc[name].get("fp32"):
            continue
        rld = P.oracle_records(O, allc[name], precision="ld")
        rf = P.oracle_records(O, allc[name], precision="ld_f32")
        fin = np.isin(rld["status"], [0, 1, 2, 7])
        d32 = np.where(fin, angles(rld["exit_dir"], rf["exit_dir"]), 0.0)
        flip = rld["status"] != rf["status"]
        f32[name] = (d32, flip)
        print(f"{name}: FP32 model: {int((d32 > F32_LISTED).sum())} rays with D32 > {F32_LISTED:g}, "
              f"{int(flip.sum())} status changes", flush=True)
    with mp.get_context("spawn").Pool(args.procs) as pool:
        res = dict(zip(jobs, pool.map(_one, jobs, chunksize=1)))
    for name in names:
        n, idx = per_case[name]
        with open(os.path.join(OUT_DIR, name + ".txt"), "w") as f:
            f.write(f"# parity case {name} (tests/parity_cases.py): {len(idx)} of {n} rays undetermined by the FP64\n"
                    "# oracle (FP64 vs long double > 1e-10), with the oracle in binary128 at the case's own step or\n"
                    "# tolerance.  Written by tests/golden/make_parity_references.py (oracle only).\n"
                    "# Columns: ray index, status, step attempts, exit direction (3), exit point (3), time of flight,\n"
                    "# weight, tile id; D64 of the exit direction (rad), exit point, time of flight and weight (their\n"
                    "# change when states are FP64 numbers).\n")
            for k in idx:
                q, qs = res[(name, int(k))]
                vals = [int(k), int(q["status"]), int(q["steps"])]
                vals += [f"{x:.17g}" for x in q["exit_dir"]] + [f"{x:.17g}" for x in q["exit_pos"]]
                vals += [f"{q['tof']:.17g}", f"{q['weight']:.17g}", int(q["tile_id"])]
                vals += [f"{float(angles(q['exit_dir'], qs['exit_dir'])):.3e}",
                         f"{float(np.abs(q['exit_pos'] - qs['exit_pos']).max()):.3e}",
                         f"{abs(float(q['tof'] - qs['tof'])):.3e}", f"{abs(float(q['weight'] - qs['weight'])):.3e}"]
                f.write(" ".join(str(x) for x in vals) + "\n")
        if name in f32:
            d32, flip = f32[name]
            sel = np.nonzero((d32 > F32_LISTED) | flip)[0]
            with open(os.path.join(OUT_DIR, name + ".f32.txt"), "w") as f:
                f.write(f"# parity case {name}: rays the FP32 model of the mixed-precision path moves by more than\n"
                        f"# {F32_LISTED:g} rad, or whose status it changes ({len(sel)} of {n}).  Long-double oracle with FP32\n"
                        "# right-hand sides and stage velocities outside r < R1 + 0.02, against the exact long-double\n"
                        "# run.  Written by tests/golden/make_parity_references.py (oracle only).\n"
                        "# Columns: ray index, D32 (rad), status changed (0/1).\n")
                for k in sel:
                    f.write(f"{int(k)} {d32[k]:.3e} {int(flip[k])}\n")
    print(f"done ({time.time() - t0:.0f} s)")
    return 0


if __name__ == "__main__":
    sys.exit(main())
