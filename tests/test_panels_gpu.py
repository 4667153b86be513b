"""Panels of the paper's figures (Figs. 1, 2 (a)-(c)): the room alone and the bare metal cylinder against
the oracle's room, and the unpolarised cloak image against the per-sample records of both polarisations."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1209_6038_gb300 import inputs

pytestmark = pytest.mark.gpu

W, H = 96, 64


@pytest.fixture(scope="module")
def ck():
    import torch
    from paper_1209_6038_gb300 import build, cloak
    build.build()
    cloak.load()
    torch.cuda.init()
    return cloak


def handle(ck, variant, elev, az=0.0):
    eye, tgt, up = inputs.camera_pose(elev, az)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, ck.FP64, 1_000_000)
    c.schedule(ck.SCHED_WAVEFRONT)
    return c, O.Camera(eye, tgt, up, 60.0, W, H)


def metal_hit(o, d, R1=0.5, halfH=1.0):
    """First hit of the ray o + s d with the closed metal cylinder r <= R1, |z| <= halfH: (point, normal)."""
    best, hit = math.inf, None
    a = d[0] ** 2 + d[1] ** 2
    b = o[0] * d[0] + o[1] * d[1]
    c = o[0] ** 2 + o[1] ** 2 - R1 * R1
    if a > 0 and b * b - a * c >= 0:
        s = (-b - math.sqrt(b * b - a * c)) / a
        if s > 0 and abs(o[2] + s * d[2]) <= halfH:
            p = o + s * d
            best, hit = s, (p, np.array([p[0], p[1], 0.0]) / math.hypot(p[0], p[1]))
    for zc, nz in ((halfH, 1.0), (-halfH, -1.0)):
        if d[2] != 0:
            s = (zc - o[2]) / d[2]
            p = o + s * d
            if 0 < s < best and p[0] ** 2 + p[1] ** 2 <= R1 * R1 and d[2] * nz < 0:
                best, hit = s, (p, np.array([0.0, 0.0, nz]))
    return hit


@pytest.mark.parametrize("elev", [0.0, 30.0])
def test_room_and_metal_panels_match_the_oracle_room(ck, elev):
    c, cam = handle(ck, 0, elev, 15.0)
    room = c.panel(ck.PANEL_ROOM).cpu().numpy().reshape(-1, 4)
    metal = c.panel(ck.PANEL_METAL).cpu().numpy().reshape(-1, 4)
    cl = O.Cloak(O.RADIAL)
    n_metal = 0
    for k in range(W * H):
        o, d = O.camera_ray(cam, k % W, k // W, 0, 1, 0)
        _, rgb = O.shade(cl, o, d)
        assert np.allclose(room[k, :3], rgb, atol=1e-6) and room[k, 3] == 1.0
        hit = metal_hit(o, d)
        if hit is None:
            assert np.allclose(metal[k, :3], rgb, atol=1e-6)
        else:
            p, n = hit
            dr = d - 2 * (d @ n) * n
            _, rgb2 = O.shade(cl, p, dr)
            n_metal += 1
            # pixels whose metal hit is within rounding of an edge may pick the other surface
            assert np.allclose(metal[k, :3], rgb2, atol=1e-6) or abs(abs(p[2]) - 1.0) < 1e-9
    assert n_metal > 100


@pytest.mark.parametrize("variant", [0, 1])
def test_unpolarised_panel_sums_the_polarisations(ck, variant):
    import torch
    c, _ = handle(ck, variant, 20.0)
    unpol = c.panel(ck.PANEL_UNPOLARIZED).cpu().numpy().reshape(-1, 4)
    img = [c.render(m).cpu().numpy().reshape(-1, 4) for m in (0, 1)]
    rec = ck.records_to_numpy(c.render_records(0))
    once = np.isin(rec["status"], [0, 7])  # missed the cylinder, or mirrored off a metal end disc
    expect = np.where(once[:, None], img[0], img[0] + img[1])
    assert once.sum() > 0 and (~once).sum() > 100
    assert np.max(np.abs(unpol - expect)) < 1e-5
    # twice more: the captured graph is replayed
    again = c.panel(ck.PANEL_UNPOLARIZED).cpu().numpy().reshape(-1, 4)
    assert np.array_equal(again, unpol)
    # and with jittered samples the panel stays between each mode's image and their sum
    u2 = c.panel(ck.PANEL_UNPOLARIZED, spp=3, seed=5).cpu().numpy().reshape(-1, 4)
    i2 = [c.render(m, spp=3, seed=5).cpu().numpy().reshape(-1, 4) for m in (0, 1)]
    assert np.all(u2 <= i2[0] + i2[1] + 1e-5) and np.all(u2 >= np.maximum(i2[0], i2[1]) - 1e-5)
