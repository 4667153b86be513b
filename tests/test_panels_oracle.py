"""Pins of the oracle's figure panels (Figs. 1, 2 (c)-(e); Sect. 4, Sect. 5): oracle.panel_image composes,
per sample, the ordinary and extraordinary light each with its own Eq. 12 factors, counting once a sample
that never enters the shell.  Pinned against the C oracle's single-polarisation images, Malus
completeness of two orthogonal polariser axes, and the bounds a polariser must respect."""
import numpy as np
import pytest

import oracle as O
from paper_1209_6038_gb300 import inputs

W, H = 31, 17  # odd width: the centre column's camera rays lie in the plane of the forward and up vectors


def cam(elev):
    eye, tgt, up = inputs.camera_pose(elev)
    return O.Camera(eye, tgt, up, 60.0, W, H)


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
@pytest.mark.parametrize("spp", [1, 3])
def test_unpolarised_panel_is_the_incoherent_sum_of_the_single_images(variant, spp):
    integ = O.Integrator(O.DP45, 1e-9)
    c = cam(20.0)
    panel = O.panel_image(variant, integ, c, "unpolarized", spp, 5)
    img = [O.render(O.Cloak(variant), integ, c, m, spp, 5)[0] for m in (O.ORDINARY, O.EXTRAORDINARY)]
    _, rec = O.render(O.Cloak(variant), integ, c, O.ORDINARY, spp, 5)
    once = np.isin(rec["status"], [O.MISSED, O.METAL_CAP]).reshape(-1, spp)
    assert once.any() and (~once).any()
    if spp == 1:  # per pixel one sample: either both images add, or the shared vacuum light counts once
        expect = np.where(once[:, :1], img[0], img[0] + img[1])
        assert np.abs(panel - expect).max() < 1e-12
    else:  # bounded by each image and by their sum
        assert np.all(panel <= img[0] + img[1] + 1e-12) and np.all(panel >= np.maximum(img[0], img[1]) - 1e-12)


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
def test_orthogonal_polarisers_add_up_to_the_unpolarised_panel(variant):
    """Malus: on the centre column the camera's right vector is across every camera ray and orthogonal to the
    up vector's part across it, so the two polariser panels add up to the unpolarised one there; elsewhere
    each polariser passes at most the unpolarised light, and a never-entering sample exactly half of it."""
    integ = O.Integrator(O.DP45, 1e-9)
    c = cam(0.0)
    unp = O.panel_image(variant, integ, c, "unpolarized")
    pr = O.panel_image(variant, integ, c, "polarizer_right")
    pu = O.panel_image(variant, integ, c, "polarizer_up")
    col = np.arange(H) * W + W // 2
    assert np.abs(pr[col] + pu[col] - unp[col]).max() < 1e-12
    assert np.all(pr <= unp + 1e-12) and np.all(pu <= unp + 1e-12)
    _, rec = O.render(O.Cloak(variant), integ, c, O.ORDINARY, 1, 0)
    never = np.isin(rec["status"], [O.MISSED, O.METAL_CAP])
    assert never.sum() > 100
    assert np.abs(pr[never] - 0.5 * unp[never]).max() < 1e-12


def test_polariser_across_the_axis_shows_the_cloaked_row():
    """Sect. 5 (after Fig. 3): through the polariser across the cylinder axis (here the camera's right
    vector at elevation 0) the extraordinary light of the centre row passes and is cloaked -- the row shows
    the room's own tiles -- while the ordinary light there is blocked.  (An even width: no pixel looks
    exactly at the axis, where the radial cloak's two waves are degenerate.)"""
    integ = O.Integrator(O.DP45, 1e-9)
    c = O.Camera((5.0, 0.0, 0.0), (0, 0, 0), (0, 0, 1), 60.0, 32, 1)  # one row, in the plane across the axis
    for variant in (O.RADIAL, O.AZIMUTHAL):
        pr = O.panel_image(variant, integ, c, "polarizer_right")
        e_only = O.render(O.Cloak(variant, analyzer=O.camera_axes(c)[0]), integ, c, O.EXTRAORDINARY, 1, 0)[0]
        o_only = O.render(O.Cloak(variant, analyzer=O.camera_axes(c)[0]), integ, c, O.ORDINARY, 1, 0)[0]
        _, rec = O.render(O.Cloak(variant), integ, c, O.ORDINARY, 1, 0)
        enters = ~np.isin(rec["status"], [O.MISSED, O.METAL_CAP])
        assert enters.sum() > 5
        assert np.abs(o_only[enters, 3]).max() < 1e-12           # ordinary light blocked
        assert np.abs(pr[enters] - e_only[enters]).max() < 1e-12  # what passes is the extraordinary light
        _, rece = O.render(O.Cloak(variant), integ, c, O.EXTRAORDINARY, 1, 0)
        room = [O.shade(O.Cloak(variant), o, d)[0] for o, d in (O.camera_ray(c, i, 0, 0, 1, 0) for i in range(32))]
        assert all(rece["tile_id"][i] == room[i] for i in np.nonzero(enters)[0])  # the room's own tiles
