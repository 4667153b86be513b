"""GPU-vs-oracle parity of the FP64 path (through the C ABI).

Bar (FP64): exit directions within 1e-9 rad of the oracle; exit points, time of
flight and Eq. 12 weights within 1e-9; statuses, room tiles and RK4 step counts
identical.  Images: RGBA within 1e-5 (FP32 colour accumulation).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1209_6038_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_DIR = 1e-9
TOL_POS = 1e-9


@pytest.fixture(scope="module")
def ck():
    import torch
    from paper_1209_6038_gb300 import build, cloak
    build.build()
    cloak.load()
    torch.cuda.init()
    return cloak


def angles(a, b):
    cr = np.linalg.norm(np.cross(a, b), axis=-1)
    dt = np.sum(a * b, axis=-1)
    return np.arctan2(cr, dt)


def compare_records(g, o, what, steps_exact=True, tol_dir=TOL_DIR, tol_pos=TOL_POS, tol_w=1e-9):
    assert g.shape == o.shape
    st_g, st_o = g["status"], o["status"]
    bad = np.nonzero(st_g != st_o)[0]
    assert len(bad) == 0, f"{what}: {len(bad)} status mismatches, e.g. idx {bad[:5]} gpu {st_g[bad[:5]]} " \
                          f"oracle {st_o[bad[:5]]}"
    assert np.array_equal(g["mode"], o["mode"])
    ok = np.isin(st_o, [0, 1, 2, 7])
    ang = angles(g["exit_dir"][ok], o["exit_dir"][ok])
    assert ang.max(initial=0) <= tol_dir, f"{what}: max exit-direction error {ang.max():.3e} rad"
    dpos = np.abs(g["exit_pos"] - o["exit_pos"]).max(axis=1)
    assert dpos.max(initial=0) <= tol_pos, f"{what}: max exit-point error {dpos.max():.3e}"
    dtof = np.abs(g["tof"] - o["tof"])
    assert dtof.max(initial=0) <= tol_pos, f"{what}: max TOF error {dtof.max():.3e}"
    dw = np.abs(g["weight"] - o["weight"])
    assert dw.max(initial=0) <= tol_w, f"{what}: max weight error {dw.max():.3e}"
    tb = np.nonzero(g["tile_id"] != o["tile_id"])[0]
    assert len(tb) == 0, f"{what}: {len(tb)} tile mismatches"
    if steps_exact:
        sb = np.nonzero(g["steps"] != o["steps"])[0]
        assert len(sb) == 0, f"{what}: {len(sb)} step-count mismatches, e.g. {g['steps'][sb[:5]]} vs " \
                             f"{o['steps'][sb[:5]]}"
    return float(ang.max(initial=0))


def gpu_trace(ck, variant, mode, rays, integ, h_or_tol, max_steps=1_000_000, test_medium=None, R1=0.5):
    import torch
    c = ck.Cloak(variant, R1=R1, R2=1.0, height=2.0)
    if test_medium:
        c.test_medium(*test_medium)
    c.integrator(integ, h_or_tol, ck.FP64, max_steps)
    out = c.trace_rays(mode, torch.from_numpy(rays))
    torch.cuda.synchronize()
    rec = ck.records_to_numpy(out)[: len(rays)]
    c.close()
    return rec


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("integ,h_or_tol", [(0, 1e-3), (1, 1e-9)])
def test_trace_rays_parity(ck, variant, mode, integ, h_or_tol):
    rays = inputs.ray_set(720, seed=11 + variant * 2 + mode, kind="mixed")
    g = gpu_trace(ck, variant, mode, rays, integ, h_or_tol)
    o = O.trace_rays(O.Cloak(variant), O.Integrator(integ, h_or_tol), mode, rays)
    compare_records(g, o, f"v{variant} m{mode} i{integ}", steps_exact=True)
    # the ray set reaches every branch the variant/mode allows
    assert (o["status"] == 0).sum() > 50 and np.isin(o["status"], [1, 2]).sum() > 300


@pytest.mark.parametrize("mode", [0, 1])
def test_test_medium_interfaces(ck, mode):
    """Homogeneous uniaxial cylinder with a tilted optic axis: entry and exit
    refraction (Sect. 3) and Eq. 12 weights for a general c-hat."""
    rays = inputs.ray_set(500, seed=5, kind="mixed")
    med = (2.2, 3.1, (0.5, -0.3, 0.81))
    g = gpu_trace(ck, 100, mode, rays, 0, 1e-2, test_medium=med, R1=0.0)
    o = O.trace_rays(O.Cloak(O.TEST_CONST, R1=0.0, eps_o=2.2, eps_e=3.1, c_hat=(0.5, -0.3, 0.81)),
                     O.Integrator(O.RK4, 1e-2), mode, rays)
    compare_records(g, o, f"test medium m{mode}")
    assert np.isin(o["status"], [1]).sum() > 200


def small_render(ck, variant, mode, integ, h_or_tol, W, H, spp, elev, seed=0, records=True):
    import torch
    eye, tgt, up = inputs.camera_pose(elev)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(integ, h_or_tol)
    img = c.render(mode, spp, seed)
    rec = c.render_records(mode, spp, seed) if records else None
    torch.cuda.synchronize()
    img = img.reshape(-1, 4).cpu().numpy().astype(np.float64)
    rec = ck.records_to_numpy(rec) if records else None
    c.close()
    return img, rec


def test_small_config_image(ck):
    """The small workload (radial, extraordinary, 128x96, 1 spp, RK4 h = 1e-3): whole image."""
    w = inputs.SMALL
    img, rec = small_render(ck, 0, 1, 0, 1e-3, w.width, w.height, 1, 0.0)
    eye, tgt, up = inputs.camera_pose(0.0)
    rgba, orec = O.render(O.Cloak(O.RADIAL), O.Integrator(O.RK4, 1e-3), O.Camera(eye, tgt, up, 60, 128, 96),
                          O.EXTRAORDINARY, 1, 0)
    compare_records(rec, orec, "small image")
    assert np.abs(img - rgba).max() < 1e-5
    assert (orec["status"] == 1).sum() > 1500


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_jittered_elevations_dp45(ck, variant, mode):
    """Both variants and polarizations, elevations 0/20/45 deg, 2 jittered samples,
    DP5(4) at tol 1e-9, 61x37 pixels (a ragged tail for 128-thread blocks)."""
    W, H, spp = 61, 37, 2
    for elev in (0.0, 20.0, 45.0):
        img, rec = small_render(ck, variant, mode, 1, 1e-9, W, H, spp, elev, seed=3)
        eye, tgt, up = inputs.camera_pose(elev)
        rgba, orec = O.render(O.Cloak(variant), O.Integrator(O.DP45, 1e-9), O.Camera(eye, tgt, up, 60, W, H),
                              mode, spp, 3)
        compare_records(rec, orec, f"v{variant} m{mode} e{elev}", steps_exact=False)
        assert np.abs(img - rgba).max() < 1e-5


def test_full_size_sampled(ck):
    """1920x1080, 4 jittered spp, DP5(4) tol 1e-9 (the full workload's launch shape),
    azimuthal cloak, extraordinary light, elevation 20 deg: a seeded sample of pixels
    against the oracle; image statistics over every pixel."""
    import torch
    w = inputs.FULL
    eye, tgt, up = inputs.camera_pose(20.0)
    c = ck.Cloak(1).camera(eye, tgt, up, 60.0, w.width, w.height).integrator(1, 1e-9)
    rec_t = c.render_records(1, w.spp, w.seed)
    img = c.render(1, w.spp, w.seed)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    pix = np.sort(rng.choice(w.width * w.height, 400, replace=False))
    rec = ck.records_to_numpy(rec_t).reshape(-1, w.spp)[pix].reshape(-1)
    rgba_g = img.reshape(-1, 4).cpu().numpy().astype(np.float64)
    rgba, orec = O.render(O.Cloak(O.AZIMUTHAL), O.Integrator(O.DP45, 1e-9),
                          O.Camera(eye, tgt, up, 60, w.width, w.height), O.EXTRAORDINARY, w.spp, w.seed, pixels=pix)
    compare_records(rec, orec, "full-size sample", steps_exact=False)
    assert np.abs(rgba_g[pix] - rgba).max() < 1e-5
    allrec = ck.records_to_numpy(rec_t)
    assert np.all(np.isfinite(rgba_g))
    assert np.isin(allrec["status"], [0, 1, 2, 3, 4, 7]).all()   # no STEP_LIMIT / SINGULAR at this tolerance
    c.close()


def test_edge_cases(ck):
    import torch
    c = ck.Cloak(0)
    # empty ray batch
    out = torch.empty(80, dtype=torch.uint8, device="cuda")
    ck.cloak_trace_rays(c.h, 1, torch.empty((0, 6), dtype=torch.float64, device="cuda"), 0, out)
    # 1x1 and odd images
    for W, H, spp in ((1, 1, 1), (7, 5, 3)):
        img, rec = small_render(ck, 0, 1, 0, 1e-3, W, H, spp, 0.0, seed=9)
        eye, tgt, up = inputs.camera_pose(0.0)
        rgba, orec = O.render(O.Cloak(0), O.Integrator(0, 1e-3), O.Camera(eye, tgt, up, 60, W, H), 1, spp, 9)
        compare_records(rec, orec, f"{W}x{H}")
    # step limit
    rays = inputs.ray_set(64, seed=2, kind="lateral")
    g = gpu_trace(ck, 1, 1, rays, 0, 1e-3, max_steps=7)
    o = O.trace_rays(O.Cloak(1), O.Integrator(0, 1e-3, 7), 1, rays)
    assert (o["status"] == 5).sum() > 30
    compare_records(g, o, "max_steps=7")
    # argument errors are reported, not launched
    with pytest.raises(ck.CloakError):
        ck.cloak_render(c.h, 1, 1, 0, torch.empty(4, device="cuda"))
    with pytest.raises(ck.CloakError):
        ck.cloak_set_integrator(c.h, 5, 1e-3)
    with pytest.raises(ck.CloakError):
        ck.cloak_camera_set(c.h, (0, 0, 0), (0, 0, 0), (0, 0, 1), 60, 8, 8)
    with pytest.raises(ck.CloakError):
        ck.cloak_create(0, 1.0, 0.5, 2.0)
    c.close()
