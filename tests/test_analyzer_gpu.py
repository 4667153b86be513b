"""The camera polariser (the paper's goggle panels, Figs. 1, 2 (d), (e)) on the GPU: ray weights against
the oracle, and the paper's observation that through the polariser across the cylinder axis the cloak
disappears along the image line of rays across the axis.  (The polariser panels themselves are compared
with the oracle's panel images in test_panels_gpu.py.)"""
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
    return u, np.cross(u, w)  # right, up


def handle(ck, variant, elev, W, H, schedule, analyzer):
    eye, tgt, up = inputs.camera_pose(elev, 10.0)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, ck.FP64, 1_000_000)
    c.schedule(schedule).analyzer(analyzer)
    return c, (eye, tgt, up)


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("variant,mode,analyzer", [(0, 1, 1), (1, 1, 1), (1, 0, 2), (0, 0, 2)])
def test_weights_match_the_oracle(ck, schedule, variant, mode, analyzer):
    W, H = 40, 29
    c, (eye, tgt, up) = handle(ck, variant, 20.0, W, H, schedule, analyzer)
    g = ck.records_to_numpy(c.render_records(mode))
    right, upv = camera_axes(eye, tgt, up)
    axis = right if analyzer == 1 else upv
    _, o = O.render(O.Cloak(variant, analyzer=tuple(axis)), O.Integrator(O.DP45, 1e-9, 1_000_000),
                    O.Camera(eye, tgt, up, 60.0, W, H), mode, spp=1, seed=0)
    same = g["status"] == o["status"]
    assert same.mean() > 0.99
    ok = same & np.isin(o["status"], [0, 1, 2, 7])
    assert np.all(o["weight"][np.isin(o["status"], [0, 7])] == 0.5)
    assert np.max(np.abs(g["weight"][ok] - o["weight"][ok])) < 1e-9
    c.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_across_axis_polariser_hides_the_cloak_on_the_central_row(ck, variant):
    """Elevation 0, odd image height: the central row's rays run across the axis.  Their e-light is
    cloaked perfectly and polarised across the axis (it passes the polariser along the camera's right
    vector), their o-light is blocked: through the polariser the row shows the bare room's own tiles,
    dimmed by the e-light's share of the transmission (the non-magnetic cloak reflects part of the light
    at its surface, so at most half)."""
    W, H = 96, 49
    eye, tgt, up = inputs.camera_pose(0.0)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-10, ck.FP64, 1_000_000)
    c.schedule(ck.SCHED_WAVEFRONT)
    room = c.panel(ck.PANEL_ROOM).cpu().numpy()
    d = c.panel(ck.PANEL_POLARIZER_RIGHT).cpu().numpy()
    unpol = c.panel(ck.PANEL_UNPOLARIZED).cpu().numpy()
    rec = ck.records_to_numpy(c.render_records(1)).reshape(H, W)
    row = H // 2
    lateral = rec["status"][row] == 1
    assert lateral.sum() > 10
    # through the polariser each cloak pixel is the bare room's colour times its weight (same tile)
    col = room[row, lateral, :3]
    assert col.min() > 1e-3
    ratio = d[row, lateral, :3] / col
    w = d[row, lateral, 3]
    assert np.max(np.abs(ratio - w[:, None])) < 1e-5
    assert np.all(w > 0.05) and np.all(w <= 0.5 + 1e-6)
    # without the polariser the same pixels are visibly disturbed (the o-light is not cloaked)
    assert np.max(np.abs(unpol[row, lateral, :3] - room[row, lateral, :3])) > 0.05
    c.close()
