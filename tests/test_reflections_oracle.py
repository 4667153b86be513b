"""Pins of the oracle's first-order reflections (the paper keeps them, Sect. 4; the double reflection
inside at the exit face, Sect. 3): energy at a face including total internal reflection, reciprocity of
the reflection coefficients (the reading that lets a camera-backward ray stand for the light), Fresnel's
closed forms in the isotropic limit, mode separation where the optic axis is the face normal, and a whole
reflected path through a homogeneous cylinder by hand."""
import math

import numpy as np
import pytest

import oracle as O

INTEG = O.Integrator(O.DP45, 1e-11, 2_000_000)


def fresnel(n1, n2, c1):
    """amplitude-free Fresnel reflectances (R_s, R_p) from index n1 to n2 at incidence cosine c1"""
    s1 = math.sqrt(max(0.0, 1 - c1 * c1))
    s2 = n1 * s1 / n2
    if s2 >= 1.0:
        return 1.0, 1.0
    c2 = math.sqrt(1 - s2 * s2)
    rs = (n1 * c1 - n2 * c2) / (n1 * c1 + n2 * c2)
    rp = (n2 * c1 - n1 * c2) / (n2 * c1 + n1 * c2)
    return rs * rs, rp * rp


def outward(cl, mode, x, n, kt):
    """the mode's wave with tangential kt travelling towards the face (these faces are mirror planes of
    the index surface: the optic axis is along or across the normal)"""
    r = O.refract_into(cl, mode, x, n, kt)
    if r is None:
        return None
    k = r[0]
    return k - 2 * np.dot(k, n) * n


def faces(rng, cl):
    for _ in range(40):
        th, z = rng.uniform(0, 2 * np.pi), rng.uniform(-0.9, 0.9)
        if rng.random() < 0.7:
            n = np.array([math.cos(th), math.sin(th), 0.0])
            x = n * 1.0 + np.array([0, 0, z])
        else:
            n = np.array([0.0, 0.0, 1.0])
            r = rng.uniform(0.55, 0.98)
            x = np.array([r * math.cos(th), r * math.sin(th), 1.0])
        u = np.cross(n, rng.normal(size=3))
        u /= np.linalg.norm(u)
        yield x, n, u


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
def test_energy_at_the_far_face_including_total_internal_reflection(variant):
    cl = O.Cloak(variant)
    rng = np.random.default_rng(3 + variant)
    n_tir = 0
    for x, n, u in faces(rng, cl):
        for mode in (O.ORDINARY, O.EXTRAORDINARY):
            for a in (0.3, 0.9, 1.3, 1.7):
                k = outward(cl, mode, x, n, a * u)
                if k is None:
                    continue
                ok, T, Ro, Re = O.transmission_out(cl, mode, x, n, k)
                assert ok
                if a > 1.0:
                    n_tir += 1
                    assert T == 0.0
                assert abs(T + Ro + Re - 1.0) < 1e-10
    assert n_tir >= 10


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
def test_reflection_coefficients_are_reciprocal(variant):
    """R(m -> m') for the wave k_m equals R(m' -> m) for the time-reversed reflected wave -k_m'."""
    cl = O.Cloak(variant)
    rng = np.random.default_rng(11 + variant)
    checked = 0
    for x, n, u in faces(rng, cl):
        for a in (0.4, 0.8, 1.2):
            kt = a * u
            for m in (O.ORDINARY, O.EXTRAORDINARY):
                km = outward(cl, m, x, n, kt)
                if km is None:
                    continue
                _, _, Ro, Re = O.transmission_out(cl, m, x, n, km)
                for m2, Rf in ((O.ORDINARY, Ro), (O.EXTRAORDINARY, Re)):
                    r2 = O.refract_into(cl, m2, x, n, kt)
                    if r2 is None:
                        continue
                    _, _, Ro2, Re2 = O.transmission_out(cl, m2, x, n, -r2[0])
                    Rb = Ro2 if m == O.ORDINARY else Re2
                    assert abs(Rf - Rb) < 1e-9 * max(1.0, Rf)
                    checked += 1
    assert checked > 100


def test_isotropic_limit_is_fresnel():
    """eps_o = eps_e = n^2 with the optic axis along z: for a face with normal z the ordinary wave is
    s-polarised and the extraordinary p-polarised; inside reflection and outside reflection are Fresnel's."""
    nidx = 1.7
    cl = O.Cloak(O.TEST_CONST, R1=0.0, eps_o=nidx ** 2, eps_e=nidx ** 2, c_hat=(0, 0, 1))
    x, nrm = np.array([0.1, 0.2, 1.0]), np.array([0.0, 0.0, 1.0])
    for a in (0.0, 0.3, 0.7, 0.95, 1.2, 1.6):
        kt = np.array([a, 0.0, 0.0])
        Rs, Rp = fresnel(nidx, 1.0, math.sqrt(max(0.0, 1 - (a / nidx) ** 2)))
        for mode, R in ((O.ORDINARY, Rs), (O.EXTRAORDINARY, Rp)):
            k = outward(cl, mode, x, nrm, kt)
            ok, T, Ro, Re = O.transmission_out(cl, mode, x, nrm, k)
            assert abs(Ro + Re - R) < 1e-10
            assert (Re if mode == O.ORDINARY else Ro) < 1e-20  # no conversion between s and p
        if a < 1.0:
            d = np.array([a, 0.0, -math.sqrt(1 - a * a)])
            t = O.transmission_in(cl, x, nrm, d)
            Rs0, Rp0 = fresnel(1.0, nidx, math.sqrt(1 - a * a))
            assert abs(t["R_s"] - Rs0) < 1e-12 and abs(t["R_p"] - Rp0) < 1e-12


def test_radial_cloak_lateral_face_separates_the_modes():
    """The radial cloak's optic axis is the lateral face's normal: an ordinary wave reflects into the
    ordinary wave alone, with Fresnel's s reflectance from n_o = 2 to vacuum."""
    cl = O.Cloak(O.RADIAL)
    th = 0.7
    n = np.array([math.cos(th), math.sin(th), 0.0])
    x = n.copy()
    for a in (0.2, 0.6, 1.1, 1.8):
        u = np.array([-math.sin(th), math.cos(th), 0.3])
        u -= np.dot(u, n) * n
        u /= np.linalg.norm(u)
        k = outward(cl, O.ORDINARY, x, n, a * u)
        ok, T, Ro, Re = O.transmission_out(cl, O.ORDINARY, x, n, k)
        Rs, _ = fresnel(2.0, 1.0, math.sqrt(1 - (a / 2.0) ** 2))
        assert abs(Ro - Rs) < 1e-10 and Re < 1e-20


def test_reflected_path_through_a_homogeneous_cylinder_by_hand():
    """Isotropic index 1.6 (optic axis z), an in-plane camera ray: refraction in (Snell), straight chord,
    mirror reflection at the far side, straight chord, refraction out.  In-plane, the ordinary wave is
    p-polarised and stays so; weight = T_p (camera side) x R_p (far side) x T_p / 2 (room light entering)."""
    nidx, R2 = 1.6, 1.0
    cl = O.Cloak(O.TEST_CONST, R1=0.0, R2=R2, eps_o=nidx ** 2, eps_e=nidx ** 2, c_hat=(0, 0, 1))
    for b in (0.1, 0.45, 0.8):
        o, d = np.array([-5.0, b, 0.0]), np.array([1.0, 0.0, 0.0])
        vac, refl = O.trace_reflections(cl, INTEG, O.ORDINARY, o, d)
        P0 = np.array([-math.sqrt(R2 * R2 - b * b), b, 0.0])
        n0 = P0 / R2
        ci = -np.dot(d, n0)
        # outer reflection of unpolarised light
        Rs0, Rp0 = fresnel(1.0, nidx, ci)
        assert abs(vac["weight"] - 0.5 * (Rs0 + Rp0)) < 1e-10
        assert np.max(np.abs(vac["exit_dir"] - (d + 2 * ci * n0))) < 1e-12
        # inside: refracted direction, chord, reflection, chord
        kt = d + ci * n0
        u = (kt - math.sqrt(nidx ** 2 - np.dot(kt, kt)) * n0) / nidx
        P1 = P0 - 2 * np.dot(P0, u) * u
        n1 = P1 / R2
        u2 = u - 2 * np.dot(u, n1) * n1
        P2 = P1 - 2 * np.dot(P1, u2) * u2
        n2 = P2 / R2
        kt2 = nidx * (u2 - np.dot(u2, n2) * n2)
        dout = kt2 + math.sqrt(1 - np.dot(kt2, kt2)) * n2
        r = refl[O.ORDINARY]
        assert r["status"] == O.EXITED
        assert np.max(np.abs(r["exit_pos"] - P2)) < 1e-9 and np.max(np.abs(r["exit_dir"] - dout)) < 1e-9
        assert abs(r["tof"] - nidx * (np.linalg.norm(P1 - P0) + np.linalg.norm(P2 - P1))) < 1e-9
        _, Rp_in = fresnel(nidx, 1.0, np.dot(u, n1))  # inside, at the far face
        _, Rp_out = fresnel(1.0, nidx, ci)             # the same angle pair at both refracting faces
        Tp = 1 - Rp_out
        assert abs(r["weight"] - Tp * Rp_in * 0.5 * Tp) < 1e-9
        assert refl[O.EXTRAORDINARY]["weight"] < 1e-20  # in-plane p light does not turn into s light


def test_rays_that_never_enter_have_no_reflections():
    cl = O.Cloak(O.RADIAL)
    vac, refl = O.trace_reflections(cl, INTEG, O.ORDINARY, (5.0, 2.0, 0.0), (-1.0, 0.0, 0.0))
    assert vac["weight"] == 0.0 and refl["weight"].sum() == 0.0 and vac["status"] == O.MISSED
    vac, refl = O.trace_reflections(cl, INTEG, O.ORDINARY, (0.2, 0.0, 5.0), (0.0, 0.0, -1.0))
    assert vac["status"] == O.METAL_CAP and vac["weight"] == 0.0


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
def test_first_order_light_never_exceeds_the_room_light(variant):
    """Per pixel, refracted plus first-order reflected light of the unpolarised image is at most the
    room light a bare pixel sees (weight 1): the camera-backward splits at each face conserve flux."""
    cam = O.Camera((4, 1, 0.8), (0, 0, 0), (0, 0, 1), 60.0, 16, 12)
    c, integ = O.Cloak(variant), O.Integrator(O.DP45, 1e-9, 1_000_000)
    _, ro = O.render(c, integ, cam, O.ORDINARY, 1, 0)
    _, re = O.render(c, integ, cam, O.EXTRAORDINARY, 1, 0)
    enters = ~np.isin(ro["status"], [O.MISSED, O.METAL_CAP])
    total = ro["weight"] + np.where(enters, re["weight"], 0.0) + O.reflections_image(c, integ, cam, 1, 0)[:, 3]
    assert np.all(total <= 1.0 + 1e-12)
    assert np.all(total[enters] > 0.3) and enters.sum() > 20
