"""First-order reflections on the GPU (the panels (c)-(e) with cloak_set_reflections): what they add to a
panel against the oracle's reflected light pixel by pixel, with and without the camera polariser, and the
flux bound of the unpolarised image."""
import numpy as np
import pytest

import oracle as O
from paper_1209_6038_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ck():
    import torch
    from paper_1209_6038_gb300 import build, cloak
    build.build()
    cloak.load()
    torch.cuda.init()
    return cloak


def camera_axes(eye, tgt, up):
    w = np.subtract(tgt, eye).astype(float)
    w /= np.linalg.norm(w)
    u = np.cross(w, up)
    u /= np.linalg.norm(u)
    return u, np.cross(u, w)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("panel", [2, 3])
def test_reflected_light_matches_the_oracle(ck, variant, panel):
    W, H = 36, 27
    eye, tgt, up = inputs.camera_pose(20.0, 4.0)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, ck.FP64, 1_000_000)
    base = c.panel(panel, 1, 0).cpu().numpy().reshape(-1, 4).astype(np.float64)
    c.reflections(True)
    full = c.panel(panel, 1, 0).cpu().numpy().reshape(-1, 4).astype(np.float64)
    c.reflections(False)
    again = c.panel(panel, 1, 0).cpu().numpy().reshape(-1, 4).astype(np.float64)
    c.close()
    assert np.array_equal(base, again)
    g = full - base
    axis = tuple(camera_axes(eye, tgt, up)[0]) if panel == 3 else (0.0, 0.0, 0.0)
    o = O.reflections_image(O.Cloak(variant, analyzer=axis), O.Integrator(O.DP45, 1e-9, 1_000_000),
                            O.Camera(eye, tgt, up, 60.0, W, H), 1, 0)
    err = np.abs(g - o).max(1)
    # float32 panels; a pixel may differ more only where a near-axis ray's status flips
    assert np.mean(err < 2e-5) > 0.99, np.sort(err)[-10:]
    assert o[:, 3].max() > 0.05


@pytest.mark.parametrize("variant", [0, 1])
def test_unpolarised_light_with_reflections_is_bounded(ck, variant):
    W, H = 64, 48
    eye, tgt, up = inputs.camera_pose(45.0, 4.0)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, ck.FP64, 1_000_000)
    c.reflections(True)
    img = c.panel(ck.PANEL_UNPOLARIZED, 2, 7).cpu().numpy().reshape(-1, 4)
    c.close()
    assert img[:, 3].max() <= 1.0 + 1e-5
    assert np.all(np.isfinite(img))
