"""Batched rendering (one persistent integration kernel for many views, CUDA graph replay) against
single-image renders of the same views, and the packet autotuner."""
import numpy as np
import pytest

from paper_1209_6038_gb300 import inputs
from test_parity_gpu import ck  # noqa: F401

pytestmark = pytest.mark.gpu

VIEWS = [  # (variant, polarization, elevation, azimuth, width, height)
    (0, 0, 0.0, 0.0, 160, 90),
    (0, 1, 20.0, 40.0, 96, 96),
    (1, 0, 45.0, 200.0, 128, 72),
    (1, 1, 10.0, 300.0, 200, 100),
    (1, 1, 0.0, 0.0, 64, 48),
    (0, 1, 55.0, 120.0, 77, 41),
]


def single(ck, variant, pol, eye, tgt, up, W, H, spp, seed, precision):
    import torch
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, precision)
    c.schedule(ck.SCHED_WAVEFRONT)
    img = c.render(pol, spp, seed)
    torch.cuda.synchronize()
    c.close()
    return img.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_single_renders(ck, precision):
    import torch
    spp, seed = 2, 17
    outs, views, refs = [], [], []
    for variant, pol, el, az, W, H in VIEWS:
        eye, tgt, up = inputs.camera_pose(el, az)
        out = torch.full((H, W, 4), -1.0, dtype=torch.float32, device="cuda")
        outs.append(out)
        views.append((variant, pol, eye, tgt, up, 60.0, out))
        refs.append(single(ck, variant, pol, eye, tgt, up, W, H, spp, seed, precision))
    h = ck.Cloak(0).integrator(ck.DP45, 1e-9, precision).schedule(ck.SCHED_WAVEFRONT)
    for rep in range(2):  # first call captures the graph, second replays it
        for o in outs:
            o.fill_(-1.0)
        ck.cloak_render_batch(h.h, views, spp, seed)
        torch.cuda.synchronize()
        for o, r in zip(outs, refs):
            got = o.cpu().numpy()
            assert np.all(np.isfinite(got)) and got.min() >= 0.0
            assert np.abs(got - r).max() <= 1e-5
    # a new seed is a new batch: captured again, matches the single render with that seed
    ck.cloak_render_batch(h.h, views[:2], spp, seed + 1)
    torch.cuda.synchronize()
    variant, pol, el, az, W, H = VIEWS[0]
    eye, tgt, up = inputs.camera_pose(el, az)
    r = single(ck, variant, pol, eye, tgt, up, W, H, spp, seed + 1, precision)
    assert np.abs(outs[0].cpu().numpy() - r).max() <= 1e-5
    h.close()


def test_batch_rejects_bad_views(ck):
    import torch
    h = ck.Cloak(0)
    out = torch.zeros((8, 8, 4), device="cuda")
    with pytest.raises(ck.CloakError):
        ck.cloak_render_batch(h.h, [(5, 0, (5, 0, 0), (0, 0, 0), (0, 0, 1), 60.0, out)], 1, 0)
    with pytest.raises(ck.CloakError):
        ck.cloak_render_batch(h.h, [(0, 0, (0, 0, 0), (0, 0, 0), (0, 0, 1), 60.0, out)], 1, 0)
    h.close()


def test_autotuner_picks_a_candidate(ck, tmp_path, monkeypatch):
    import torch
    from paper_1209_6038_gb300 import autotune
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "cache.json"))
    eye, tgt, up = inputs.camera_pose(20.0)
    c = ck.Cloak(1).camera(eye, tgt, up, 60.0, 160, 90).integrator(ck.DP45, 1e-9).schedule(ck.SCHED_WAVEFRONT)
    out = torch.empty((90, 160, 4), device="cuda")
    with pytest.raises(ck.CloakError):  # more threads per block than the persistent kernel is built for
        c.schedule(ck.SCHED_WAVEFRONT, 256)
    best, times = autotune.tune_packet(c, lambda: c.render(1, 1, 0, out=out), key="test", candidates=(64, 128))
    assert best in (64, 128) and set(times) == {64, 128}
    best2, _ = autotune.tune_packet(c, lambda: c.render(1, 1, 0, out=out), key="test", candidates=(64, 128))
    assert best2 == best  # from the cache
    c.close()
