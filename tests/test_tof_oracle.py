"""Pins of the oracle's time-of-flight difference images (Sect. 4; the TOF images of Ref. [10]): room
distances by geometry, rays that miss, the metal end disc, the radial cloak's ordinary rays (straight
lines in the index-2 medium, mirrored at the metal cylinder: a closed form), and the paper's expectation
that in-plane extraordinary light arrives exactly when it would without the cylinder."""
import math

import numpy as np

import oracle as O

INTEG = O.Integrator(O.DP45, 1e-11, 2_000_000)


def test_room_distance_by_geometry():
    c = O.Cloak(O.RADIAL)  # H = 2: floor at z = -1, ceiling at z = 9, walls at |x|, |y| = 10
    assert O.room_distance(c, (0, 0, 0), (1, 0, 0)) == 10.0
    assert O.room_distance(c, (0, 0, 0), (0, -1, 0)) == 10.0
    assert O.room_distance(c, (0, 0, 0), (0, 0, -1)) == 1.0
    assert O.room_distance(c, (0, 0, 0), (0, 0, 1)) == 9.0
    s = 1 / math.sqrt(2)
    assert abs(O.room_distance(c, (0, 0, 0), (s, s, 0)) - 10 * math.sqrt(2)) < 1e-12
    assert abs(O.room_distance(c, (3, -2, 0.5), (0.6, 0.0, -0.8)) - 1.5 / 0.8) < 1e-12  # floor before the wall


def test_a_missing_ray_has_no_delay():
    c = O.Cloak(O.AZIMUTHAL)
    o, d = np.array([5.0, 2.0, 0.3]), np.array([-1.0, 0.0, 0.0])
    for mode in (O.ORDINARY, O.EXTRAORDINARY):
        rec, _ = O.trace_ray(c, INTEG, mode, o, d)
        assert rec["status"] == O.MISSED
        assert O.tof_difference(c, o, d, rec) == 0.0


def test_metal_end_disc():
    c = O.Cloak(O.RADIAL)
    o, d = np.array([0.2, 0.0, 5.0]), np.array([0.0, 0.0, -1.0])
    rec, _ = O.trace_ray(c, INTEG, O.EXTRAORDINARY, o, d)
    assert rec["status"] == O.METAL_CAP
    # down 4 to the disc at z = 1, up 8 to the ceiling at z = 9; without the cylinder: down 6 to the floor
    assert abs(O.tof_difference(c, o, d, rec) - (4 + 8 - 6)) < 1e-12


def test_radial_ordinary_rays_closed_form():
    """In the radial cloak the ordinary index is sqrt(K) = 2 everywhere: an in-plane ray refracts by
    Snell's law, runs straight at speed 1/2 to the metal cylinder, mirrors and leaves symmetrically."""
    R1, R2 = 0.5, 1.0
    n = 2.0
    c = O.Cloak(O.RADIAL, R1, R2)
    for b in (0.15, 0.4, 0.7, 0.93):
        o, d = np.array([-5.0, b, 0.0]), np.array([1.0, 0.0, 0.0])
        rec, _ = O.trace_ray(c, INTEG, O.ORDINARY, o, d)
        assert rec["status"] == O.HIT_METAL_EXITED
        # entry point and refracted direction (tangential wave-vector component conserved)
        P1 = np.array([-math.sqrt(R2 * R2 - b * b), b, 0.0])
        nrm = P1 / R2
        kt = d - np.dot(d, nrm) * nrm
        q = math.sqrt(n * n - np.dot(kt, kt))
        k = kt - q * nrm
        u = k / np.linalg.norm(k)
        # straight to r = R1
        B = np.dot(P1, u)
        s1 = -B - math.sqrt(B * B - (np.dot(P1, P1) - R1 * R1))
        P2 = P1 + s1 * u
        m = P2 / R1
        u2 = u - 2 * np.dot(u, m) * m
        B2 = np.dot(P2, u2)
        s2 = -B2 + math.sqrt(B2 * B2 - (np.dot(P2, P2) - R2 * R2))
        P3 = P2 + s2 * u2
        n3 = P3 / R2
        kt3 = n * u2 - np.dot(n * u2, n3) * n3
        d3 = kt3 + math.sqrt(1 - np.dot(kt3, kt3)) * n3
        t = np.linalg.norm(P1 - o) + n * (s1 + s2) + O.room_distance(c, P3, d3)
        expect = t - O.room_distance(c, o, d)
        assert np.max(np.abs(rec["exit_pos"] - P3)) < 1e-9
        assert abs(O.tof_difference(c, o, d, rec) - expect) < 1e-9


def test_in_plane_extraordinary_light_arrives_on_time():
    """The horizontal centre row of a level camera (odd image height) sees the cloak with in-plane rays:
    their extraordinary light is perfectly cloaked, so its TOF difference vanishes; with the polariser
    across the cylinder axis the ordinary light is blocked there and the pixel's TOF equals the bare room's."""
    W, H = 24, 13
    for variant in (O.RADIAL, O.AZIMUTHAL):
        cam = O.Camera((5, 0, 0), (0, 0, 0), (0, 0, 1), 60.0, W, H)
        row = np.arange(6 * W, 7 * W)
        img = O.tof_image(O.Cloak(variant), INTEG, cam, 1, 0, pixels=row)
        hit = img[:, 3] < 1.0
        assert hit.sum() >= 6
        assert np.max(np.abs(img[:, 2])) < 1e-9
        assert np.max(np.abs(img[hit, 1])) > 0.1  # the ordinary light is delayed (or advanced)
        pol = O.tof_image(O.Cloak(variant, analyzer=(0.0, 1.0, 0.0)), INTEG, cam, 1, 0, pixels=row)
        assert np.max(np.abs(pol[:, 0])) < 1e-9


def test_tof_image_weights_match_the_unpolarised_alpha():
    cam = O.Camera((4, 1, 1.2), (0, 0, 0), (0, 0, 1), 60.0, 12, 9)
    c = O.Cloak(O.RADIAL)
    img = O.tof_image(c, INTEG, cam, 2, 5)
    ro, rec_o = O.render(c, INTEG, cam, O.ORDINARY, 2, 5)
    re, rec_e = O.render(c, INTEG, cam, O.EXTRAORDINARY, 2, 5)
    enters = ~np.isin(rec_o["status"], [O.MISSED, O.METAL_CAP])
    alpha = (rec_o["weight"] + np.where(enters, rec_e["weight"], 0.0)).reshape(-1, 2).mean(1)
    assert np.allclose(img[:, 3], alpha, rtol=0, atol=1e-15)
    assert np.any(enters) and np.any(~enters)
