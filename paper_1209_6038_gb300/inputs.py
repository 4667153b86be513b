"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method itself: it only lays out ray
sets, camera poses and workload descriptions.  The paper's own scenery is not
available; a procedural checkerboard room stands in for it, and the geometry
keeps the paper's ratio a/b = 0.5 (a = 5 cm, b = 10 cm in Sect. 4) as
R1 = 0.5, R2 = 1.0 with height 2.0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RADIAL, AZIMUTHAL = 0, 1
ORDINARY, EXTRAORDINARY = 0, 1
GEOMETRY = dict(R1=0.5, R2=1.0, H=2.0)
CAMERA_DISTANCE = 5.0


def camera_pose(elevation_deg: float = 0.0, azimuth_deg: float = 0.0, distance: float = CAMERA_DISTANCE):
    """Eye on a sphere around the cloak centre, looking at the origin, up = +z."""
    e, a = math.radians(elevation_deg), math.radians(azimuth_deg)
    eye = (distance * math.cos(e) * math.cos(a), distance * math.cos(e) * math.sin(a), distance * math.sin(e))
    return eye, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0)


@dataclass(frozen=True)
class Workload:
    """One rendering workload: every (variant, polarization, elevation) image."""
    name: str
    variants: tuple
    pols: tuple
    elevations: tuple
    width: int
    height: int
    spp: int
    integrator: str          # "rk4" (fixed h) or "dp45" (adaptive, tolerance)
    h_or_tol: float
    hfov_deg: float = 60.0
    seed: int = 0
    max_steps: int = 1_000_000
    extra: dict = field(default_factory=dict)

    @property
    def images(self):
        return [(v, p, e) for v in self.variants for p in self.pols for e in self.elevations]

    @property
    def rays_per_image(self):
        return self.width * self.height * self.spp

    @property
    def rays(self):
        return self.rays_per_image * len(self.images)


# small: radial cloak, extraordinary light, 128x96, 1 spp, RK4 h = 1e-3
SMALL = Workload("radial e-pol 128x96 1spp RK4 h=1e-3", (RADIAL,), (EXTRAORDINARY,), (0.0,), 128, 96, 1,
                 "rk4", 1e-3)
# full: both variants x both polarizations x elevations 0/20/45 deg, 1920x1080, 4 jittered spp, DP5(4) tol 1e-9
FULL = Workload("2 variants x 2 pols x elev {0,20,45} 1920x1080 4spp DP45 tol=1e-9", (RADIAL, AZIMUTHAL),
                (ORDINARY, EXTRAORDINARY), (0.0, 20.0, 45.0), 1920, 1080, 4, "dp45", 1e-9)

# surrogate: the same twelve views at 3840x2160, 1 spp; the learned surrogate is trained on 10^7 rays that
# the FP64 DP5(4) integrator traces (entry points uniform on the lateral surface, directions
# cosine-weighted about the inward normal), the integrator handles the rest
SURROGATE = Workload("2 variants x 2 pols x elev {0,20,45} 3840x2160 1spp surrogate + DP45 tol=1e-9 FP64 fallback",
                     (RADIAL, AZIMUTHAL), (ORDINARY, EXTRAORDINARY), (0.0, 20.0, 45.0), 3840, 2160, 1, "dp45", 1e-9,
                     extra={"train_rays": 10_000_000, "train_seed": 0, "gate_log10_err": -3.0})


def ray_set(n: int, seed: int, kind: str = "mixed", R2: float = 1.0, H: float = 2.0, distance: float = 3.0):
    """(n, 6) array of ray origins and unit directions (x, y, z, dx, dy, dz)
    starting outside the cylinder r <= R2, |z| <= H/2.

    kinds: "lateral" (aimed at the side face), "inplane" (z = dz = 0),
    "grazing" (impact parameter within 1e-2 of R2), "near_axis" (impact
    parameter below 1e-2 -- close to the singular inner radius), "cap" (from
    above or below through an end face), "miss", "mixed" (all of them)."""
    rng = np.random.default_rng(seed)
    if kind == "mixed":
        kinds = ["lateral", "inplane", "grazing", "near_axis", "cap", "miss"]
        parts = np.array_split(np.arange(n), len(kinds))
        out = np.zeros((n, 6))
        for ik, (k, idx) in enumerate(zip(kinds, parts)):
            if len(idx):
                out[idx] = ray_set(len(idx), seed * 7919 + ik + 1, k, R2, H, distance)
        return out[rng.permutation(n)]
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    if kind == "cap":
        top = rng.uniform(size=n) < 0.5
        sgn = np.where(top, 1.0, -1.0)
        rad = R2 * np.sqrt(rng.uniform(0.0, 1.0, n)) * 0.999
        ang = rng.uniform(0, 2 * math.pi, n)
        tgt = np.stack([rad * np.cos(ang), rad * np.sin(ang), sgn * 0.5 * H], 1)
        th = np.radians(rng.uniform(0.0, 60.0, n))
        az = rng.uniform(0, 2 * math.pi, n)
        dirs = np.stack([np.sin(th) * np.cos(az), np.sin(th) * np.sin(az), -sgn * np.cos(th)], 1)
        org = tgt - 2.0 * dirs
        return np.concatenate([org, dirs], 1)
    if kind == "lateral":
        b = rng.uniform(-0.98, 0.98, n) * R2
        zt = rng.uniform(-0.4, 0.4, n) * H
    elif kind == "inplane":
        b = rng.uniform(-0.98, 0.98, n) * R2
        zt = np.zeros(n)
    elif kind == "grazing":
        b = np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0) * R2 * (1.0 - 10.0 ** rng.uniform(-5, -2, n))
        zt = rng.uniform(-0.3, 0.3, n) * H
    elif kind == "near_axis":
        b = np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0) * R2 * 10.0 ** rng.uniform(-4, -2, n)
        zt = rng.uniform(-0.3, 0.3, n) * H
    elif kind == "miss":
        b = np.where(rng.uniform(size=n) < 0.5, 1.0, -1.0) * R2 * rng.uniform(1.05, 2.0, n)
        zt = rng.uniform(-0.4, 0.4, n) * H
    else:
        raise ValueError(kind)
    z0 = np.zeros(n) if kind == "inplane" else rng.uniform(-0.3, 0.3, n) * H
    # origin on a circle of radius `distance`, target (0, b, zt) in the frame rotated by phi
    ox, oy = distance * np.cos(phi), distance * np.sin(phi)
    tx, ty = -b * np.sin(phi), b * np.cos(phi)
    d = np.stack([tx - ox, ty - oy, zt - z0], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return np.concatenate([np.stack([ox, oy, z0], 1), d], 1)


def sample_pixels(w: Workload, img_index: int, n: int, seed: int = 12345):
    """Seeded sample of n distinct pixels (flat indices j * width + i, sorted) of image img_index of w: the
    pixels whose rays are checked against the oracle."""
    rng = np.random.default_rng(seed + img_index)
    return np.sort(rng.choice(w.width * w.height, n, replace=False))


BATCH_RESOLUTIONS = ((256, 256), (1024, 768), (1920, 1080), (3840, 2160))


def batched_views(n_poses: int = 64, seed: int = 0, resolutions=BATCH_RESOLUTIONS, hfov_deg: float = 60.0):
    """Seeded orbit of camera poses (azimuth ~ U[0, 360) deg, elevation ~ U[0, 60) deg, distance 5),
    each at a resolution drawn uniformly from `resolutions`, rendered for both cloaks and both
    polarizations: a list of (variant, polarization, eye, target, up, hfov_deg, width, height)."""
    rng = np.random.default_rng(seed)
    views = []
    for _ in range(n_poses):
        az = rng.uniform(0.0, 360.0)
        el = rng.uniform(0.0, 60.0)
        W, H = resolutions[int(rng.integers(len(resolutions)))]
        eye, tgt, up = camera_pose(el, az)
        for v in (RADIAL, AZIMUTHAL):
            for p in (ORDINARY, EXTRAORDINARY):
                views.append((v, p, eye, tgt, up, hfov_deg, W, H))
    return views
