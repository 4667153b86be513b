"""Time-of-flight difference images (Sect. 4 after Ref. [10]) on the GPU: the TOF panel against the
oracle's TOF images pixel by pixel, and the paper's expectation on the centre row of a level camera
(extraordinary light arrives exactly when it would without the cylinder; through the polariser across
the cylinder axis the whole pixel does)."""
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
@pytest.mark.parametrize("analyzer", [0, 1])
def test_tof_panel_matches_the_oracle(ck, variant, analyzer):
    W, H, spp = 40, 29, 2
    eye, tgt, up = inputs.camera_pose(20.0, 10.0)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, ck.FP64, 1_000_000)
    c.analyzer(analyzer)
    g = c.panel(ck.PANEL_TOF, spp, 3).cpu().numpy().reshape(-1, 4).astype(np.float64)
    c.close()
    axis = tuple(camera_axes(eye, tgt, up)[0]) if analyzer == 1 else (0.0, 0.0, 0.0)
    o = O.tof_image(O.Cloak(variant, analyzer=axis), O.Integrator(O.DP45, 1e-9, 1_000_000),
                    O.Camera(eye, tgt, up, 60.0, W, H), spp, 3)
    assert np.max(np.abs(g[:, 3] - o[:, 3])) < 1e-5
    err = np.abs(g[:, :3] - o[:, :3]).max(1)
    # float32 output of FP64 sums; a pixel may differ more only where a near-axis ray's status flips
    assert np.mean(err < 1e-5) > 0.995
    # pixels whose samples all miss the cylinder: no delay, exactly (metal end discs also keep the full
    # weight, but with a delay); a grazing sample may enter on one side and miss on the other
    miss = (o[:, 3] == (0.5 if analyzer else 1.0)) & np.all(o[:, :3] == 0.0, axis=1)
    zero = np.all(g[miss, :3] == 0.0, axis=1)
    assert miss.sum() > 100 and zero.mean() > 0.995, g[miss][~zero]
    assert np.max(np.abs(o[:, 1])) > 0.1  # the ordinary light is delayed somewhere


@pytest.mark.parametrize("variant", [0, 1])
def test_tof_centre_row_of_a_level_camera(ck, variant):
    W, H = 64, 41
    eye, tgt, up = (5.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-10, ck.FP64, 1_000_000)
    row = c.panel(ck.PANEL_TOF, 1, 0).cpu().numpy()[H // 2].astype(np.float64)
    hit = row[:, 3] < 1.0
    assert hit.sum() >= 10
    assert np.max(np.abs(row[:, 2])) < 1e-6        # extraordinary light: no delay (perfect cloaking)
    assert np.max(np.abs(row[hit, 1])) > 0.1        # ordinary light: delayed or advanced
    c.analyzer(ck.ANALYZER_RIGHT)                   # the paper's "vertical" goggles
    pol = c.panel(ck.PANEL_TOF, 1, 0).cpu().numpy()[H // 2].astype(np.float64)
    assert np.max(np.abs(pol[:, 0])) < 1e-6
    c.close()


def test_tof_panel_needs_the_integrator(ck):
    import torch
    c = ck.Cloak(ck.RADIAL).camera((5, 0, 0), (0, 0, 0), (0, 0, 1), 60.0, 8, 6)
    c.integrator(ck.DP45, 1e-9, ck.SURROGATE)
    out = torch.empty((6, 8, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ck.CloakError):
        c.panel(ck.PANEL_TOF, 1, 0, out=out)
    c.close()
