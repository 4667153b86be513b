"""The seeded inputs of the GPU parity tests, named, so that the reference script in tests/golden/ and the
tests build the same rays.  Holds no arithmetic of the method: ray sets, cameras and integrator settings.

A case is a ray set (origins and directions through cloak_trace_rays / orc_trace_rays) or a camera render
(cloak_render_records / orc_render over all pixels or a pixel subset).
"""
from __future__ import annotations

import numpy as np

from paper_1209_6038_gb300 import inputs

RK4, DP45 = 0, 1
GEOMETRIES = ((0.05, 1.0, 2.0), (0.9, 1.0, 2.0), (1.2, 3.0, 0.7))
TEST_MEDIUM = (2.2, 3.1, (0.5, -0.3, 0.81))


def _geom_name(g):
    return "R1_%g_R2_%g_H_%g" % g


def cases():
    """name -> spec (a dict).  Ray sets: kind "rays", variant, mode, integ, h_or_tol, max_steps, geometry,
    rays (n x 6).  Renders: kind "render", variant, mode, integ, h_or_tol, geometry, elevation, width, height,
    spp, seed, pixels (None: every pixel)."""
    out = {}
    for v in (0, 1):
        for m in (0, 1):
            for integ, h in ((RK4, 1e-3), (DP45, 1e-9)):
                out[f"rays_v{v}_m{m}_i{integ}"] = dict(kind="rays", variant=v, mode=m, integ=integ, h_or_tol=h,
                                                      max_steps=1_000_000, geometry=(0.5, 1.0, 2.0),
                                                      rays=lambda v=v, m=m: inputs.ray_set(720, seed=11 + v * 2 + m))
    for m in (0, 1):
        out[f"test_medium_m{m}"] = dict(kind="rays", variant=100, mode=m, integ=RK4, h_or_tol=1e-2, max_steps=1_000_000,
                                        geometry=(0.0, 1.0, 2.0), medium=TEST_MEDIUM,
                                        rays=lambda: inputs.ray_set(500, seed=5))
    out["rays_step_limit"] = dict(kind="rays", variant=1, mode=1, integ=RK4, h_or_tol=1e-3, max_steps=7,
                                  geometry=(0.5, 1.0, 2.0), rays=lambda: inputs.ray_set(64, seed=2, kind="lateral"))
    for g in GEOMETRIES:
        for v in (0, 1):
            for m in (0, 1):
                out[f"geom_{_geom_name(g)}_v{v}_m{m}"] = dict(
                    kind="rays", variant=v, mode=m, integ=DP45, h_or_tol=1e-9, max_steps=2_000_000, geometry=g,
                    rays=lambda g=g, v=v, m=m: inputs.ray_set(240, seed=31 + 2 * v + m, R2=g[1], H=g[2],
                                                              distance=3.0 * g[1]))
    w = inputs.SMALL
    out["render_small"] = dict(kind="render", variant=0, mode=1, integ=RK4, h_or_tol=1e-3, geometry=(0.5, 1.0, 2.0),
                               elevation=0.0, width=w.width, height=w.height, spp=1, seed=0, pixels=None)
    for v in (0, 1):
        for m in (0, 1):
            for e in (0.0, 20.0, 45.0):
                out[f"render_jitter_v{v}_m{m}_e{int(e)}"] = dict(
                    kind="render", variant=v, mode=m, integ=DP45, h_or_tol=1e-9, geometry=(0.5, 1.0, 2.0),
                    elevation=e, width=61, height=37, spp=2, seed=3, pixels=None)
            out[f"render_squat_v{v}_m{m}"] = dict(kind="render", variant=v, mode=m, integ=DP45, h_or_tol=1e-9,
                                                  geometry=(1.2, 3.0, 0.7), elevation=20.0, width=64, height=48,
                                                  spp=2, seed=3, pixels=None)
    for W, H, spp in ((1, 1, 1), (7, 5, 3)):
        out[f"render_edge_{W}x{H}x{spp}"] = dict(kind="render", variant=0, mode=1, integ=RK4, h_or_tol=1e-3,
                                                 geometry=(0.5, 1.0, 2.0), elevation=0.0, width=W, height=H, spp=spp,
                                                 seed=9, pixels=None)
    # the mixed-precision path's cases (FP32 right-hand sides): also given D32, the exit-direction change of
    # the oracle's FP32 model (tests/golden/make_parity_references.py)
    for v in (0, 1):
        for m in (0, 1):
            for e in (0.0, 20.0, 45.0):
                out[f"mixed_v{v}_m{m}_e{int(e)}"] = dict(kind="render", variant=v, mode=m, integ=DP45, h_or_tol=1e-9,
                                                         geometry=(0.5, 1.0, 2.0), elevation=e, width=96, height=54,
                                                         spp=2, seed=7, pixels=None, fp32=True)
    for g in ((0.9, 1.0, 2.0), (1.2, 3.0, 0.7)):
        for v in (0, 1):
            out[f"mixed_geom_{_geom_name(g)}_v{v}"] = dict(kind="render", variant=v, mode=1, integ=DP45,
                                                           h_or_tol=1e-9, geometry=g, elevation=20.0, width=64,
                                                           height=48, spp=2, seed=4, pixels=None, fp32=True)
    full = inputs.FULL
    out["mixed_full_pixels"] = dict(kind="render", variant=1, mode=1, integ=DP45, h_or_tol=1e-9,
                                    geometry=(0.5, 1.0, 2.0), elevation=20.0, width=full.width, height=full.height,
                                    spp=full.spp, seed=full.seed, fp32=True,
                                    pixels=lambda: np.sort(np.random.default_rng(1).choice(
                                        full.width * full.height, 2000, replace=False)))
    out["render_small"]["fp32"] = True  # the small workload runs on the mixed path too
    out["render_full_sampled"] = dict(kind="render", variant=1, mode=1, integ=DP45, h_or_tol=1e-9,
                                      geometry=(0.5, 1.0, 2.0), elevation=20.0, width=full.width, height=full.height,
                                      spp=full.spp, seed=full.seed,
                                      pixels=lambda: np.sort(np.random.default_rng(0).choice(
                                          full.width * full.height, 400, replace=False)))
    return out


def materialise(spec):
    """The spec with its lazily built arrays (rays, pixels) evaluated."""
    s = dict(spec)
    for k in ("rays", "pixels"):
        if callable(s.get(k)):
            s[k] = s[k]()
    return s


def oracle_records(O, spec, precision="f64", tol=None, nthreads=None):
    """Records of a case from the oracle (precision "f64", or an extended build: "ld", "q", "q_s64",
    "ld_f32"); tol overrides the case's step / tolerance."""
    s = materialise(spec)
    R1, R2, H = s["geometry"]
    if s["variant"] == 100:
        eo, ee, ch = s["medium"]
        cl = O.Cloak(O.TEST_CONST, R1=R1, R2=R2, H=H, eps_o=eo, eps_e=ee, c_hat=ch)
    else:
        cl = O.Cloak(s["variant"], R1=R1, R2=R2, H=H)
    integ = O.Integrator(s["integ"], s["h_or_tol"] if tol is None else tol, s.get("max_steps", 1_000_000))
    if s["kind"] == "rays":
        return O.trace_rays(cl, integ, s["mode"], s["rays"], nthreads=nthreads, precision=precision)
    eye, tgt, up = inputs.camera_pose(s["elevation"])
    cam = O.Camera(eye, tgt, up, 60.0, s["width"], s["height"])
    return O.render(cl, integ, cam, s["mode"], s["spp"], s["seed"], pixels=s["pixels"], nthreads=nthreads,
                    precision=precision)[1]
