"""Pins of the polarisation analyser ("goggles", Figs. 1, 2 (d), (e)) in the oracle against the paper's
Sect. 5 account (Fig. 3).  The paper's images show the cylinder axis horizontal; here it is vertical
(+z), so its "vertical plane" is the plane across the axis and its "horizontal plane" a plane containing
the axis: extraordinary light in the plane across the axis is polarised within that plane for both
cloaks; in a plane containing the axis the radial cloak keeps it in the plane while the azimuthal cloak
turns it across the plane; ordinary light is the complement.  And Malus's law."""
import math

import numpy as np
import pytest

import oracle as O

Z = np.array([0.0, 0.0, 1.0])


def exit_fraction(variant, mode, phi, d, axis):
    """A camera ray d meets the lateral surface at azimuth phi, height 0; the light that leaves there
    towards the camera in `mode`: the fraction of it passing a polariser with the given axis."""
    x = np.array([math.cos(phi), math.sin(phi), 0.0])
    n = np.array([x[0], x[1], 0.0])  # outward normal
    cl = O.Cloak(variant, analyzer=tuple(axis))
    kt = d - (d @ n) * n
    k0, _ = O.refract_into(cl, mode, x, n, kt)
    return O.analyzer_fraction(cl, mode, x, n, -k0)


@pytest.mark.parametrize("beta", [0.3, -0.7, 1.1])
def test_rays_across_the_axis(beta):
    """Both cloaks: e-light polarised within the plane across the axis (the perfectly cloaked set)."""
    phi = 0.4
    rh, th = np.array([math.cos(phi), math.sin(phi), 0]), np.array([-math.sin(phi), math.cos(phi), 0])
    d = -math.cos(beta) * rh + math.sin(beta) * th  # in the plane across the axis, not along the normal
    across = np.cross(Z, d)  # in that plane, across the ray
    for variant in (O.RADIAL, O.AZIMUTHAL):
        fe_z = exit_fraction(variant, O.EXTRAORDINARY, phi, d, Z)
        fe_a = exit_fraction(variant, O.EXTRAORDINARY, phi, d, across)
        fo_z = exit_fraction(variant, O.ORDINARY, phi, d, Z)
        assert abs(fe_z + fe_a - 1) < 1e-12
        assert fe_a > 1 - 1e-12 and fo_z > 1 - 1e-12


@pytest.mark.parametrize("alpha", [0.25, -0.6])
def test_rays_in_a_plane_containing_the_axis(alpha):
    """Radial cloak: e-light polarised in that plane; azimuthal cloak: across it (along theta-hat)."""
    phi = 1.3
    rh = np.array([math.cos(phi), math.sin(phi), 0])
    d = -math.cos(alpha) * rh + math.sin(alpha) * Z  # the plane spanned by the axis and the normal
    inplane = Z - (Z @ d) * d  # in that plane, across the ray
    for variant, e_in_plane in ((O.RADIAL, True), (O.AZIMUTHAL, False)):
        fe = exit_fraction(variant, O.EXTRAORDINARY, phi, d, inplane)
        fo = exit_fraction(variant, O.ORDINARY, phi, d, inplane)
        if e_in_plane:
            assert fe > 1 - 1e-12 and fo < 1e-12
        else:
            assert fe < 1e-12 and fo > 1 - 1e-12


def test_malus_completeness_and_unpolarised_rays():
    rng = np.random.default_rng(3)
    for _ in range(20):
        phi = rng.uniform(0, 2 * math.pi)
        rh, th = np.array([math.cos(phi), math.sin(phi), 0]), np.array([-math.sin(phi), math.cos(phi), 0])
        d = -rh * rng.uniform(0.3, 1) + th * rng.uniform(-0.6, 0.6) + Z * rng.uniform(-0.6, 0.6)
        d /= np.linalg.norm(d)
        for variant in (O.RADIAL, O.AZIMUTHAL):
            for mode in (O.ORDINARY, O.EXTRAORDINARY):
                # two orthogonal axes across the vacuum wave leaving towards the camera (along -d)
                a1 = np.cross(d, Z)
                a1 /= np.linalg.norm(a1)
                a2 = np.cross(d, a1)
                f1 = exit_fraction(variant, mode, phi, d, a1)
                f2 = exit_fraction(variant, mode, phi, d, a2)
                assert 0 <= f1 <= 1 and abs(f1 + f2 - 1) < 1e-12
    # rays that never enter: unpolarised room light, half passes
    cam = O.Camera((5, 0, 3), (0, 0, 0), (0, 0, 1), 60, 8, 6)
    o, d = O.camera_ray(cam, 0, 0, 0, 1, 0)
    rec, _ = O.trace_ray(O.Cloak(O.RADIAL, analyzer=(0, 0, 1)), O.Integrator(O.RK4, 1e-3), 1, o, d)
    assert rec["status"] == 0 and rec["weight"] == 0.5


def test_trace_weight_carries_the_fraction():
    """The ray weight with an analyser is the Eq. 12 weight times the exit polariser fraction."""
    integ = O.Integrator(O.DP45, 1e-10, 1_000_000)
    o = np.array([4.0, 0.3, 0.2])
    d = np.array([0.0, 0.45, 0.0]) - o  # impact parameter about 0.45: the ray enters and leaves laterally
    d /= np.linalg.norm(d)
    for variant in (O.RADIAL, O.AZIMUTHAL):
        for mode in (O.ORDINARY, O.EXTRAORDINARY):
            r0, _ = O.trace_ray(O.Cloak(variant), integ, mode, o, d)
            a1 = np.cross(d, Z)
            a1 /= np.linalg.norm(a1)
            a2 = np.cross(d, a1)
            r1, _ = O.trace_ray(O.Cloak(variant, analyzer=tuple(a1)), integ, mode, o, d)
            r2, _ = O.trace_ray(O.Cloak(variant, analyzer=tuple(a2)), integ, mode, o, d)
            assert r0["status"] in (1, 2)
            assert abs(r1["weight"] + r2["weight"] - r0["weight"]) < 1e-12
            assert np.array_equal(r1["exit_dir"], r0["exit_dir"])
