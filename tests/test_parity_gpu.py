"""GPU-vs-oracle parity of the FP64 path (through the C ABI).

Bar (FP64): exit directions within 1e-9 rad of the oracle, exit points, times of
flight and Eq. 12 weights within 1e-9, statuses, room tiles and RK4 step counts
identical; images (FP32 colour accumulation) within 1e-5.

Where FP64 arithmetic itself does not determine a result to that level, the bar
widens to what it does determine.  For every ray the oracle is re-run on inputs
perturbed by 1e-13 (ray origins and directions, or the camera): the change of
its own output is that ray's spread, and a GPU value may differ from the oracle
by 1e-9 + 10 x spread (four perturbations for ray sets, three for images).  Rays whose status flips under the perturbation (coarse
steps near r = R1) are checked for validity only, and their share is bounded.
A room-tile mismatch is accepted only where the oracle's hit point lies on a tile
edge (pixel-centre rays of a camera at z = 0 hit the floor at rational points).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1209_6038_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_DIR = 1e-9      # FP64 exit-direction bar (rad)
TOL_ABS = 1e-9      # exit point, time of flight, weight
KAPPA = 10.0        # multiple of the oracle's own spread that a difference may reach
PERTURB = 1e-13     # size of the input perturbation that measures that spread


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


def perturb_rays(rays, k):
    rng = np.random.default_rng(1000 + k)
    pr = rays.copy()
    pr[:, :3] += PERTURB * rng.normal(size=(len(rays), 3))
    d = pr[:, 3:] + PERTURB * rng.normal(size=(len(rays), 3))
    pr[:, 3:] = d / np.linalg.norm(d, axis=1, keepdims=True)
    return pr


def spread_of(base, others):
    """Per-ray change of the oracle's own output under 1e-13 input perturbations:
    the part of each result that FP64 arithmetic does not determine."""
    sp = dict(dir=np.zeros(len(base)), pos=np.zeros(len(base)), tof=np.zeros(len(base)), w=np.zeros(len(base)),
              unstable=np.zeros(len(base), bool), tiles=[base["tile_id"]])
    for o2 in others:
        sp["dir"] = np.maximum(sp["dir"], angles(o2["exit_dir"], base["exit_dir"]))
        sp["pos"] = np.maximum(sp["pos"], np.abs(o2["exit_pos"] - base["exit_pos"]).max(1))
        sp["tof"] = np.maximum(sp["tof"], np.abs(o2["tof"] - base["tof"]))
        sp["w"] = np.maximum(sp["w"], np.abs(o2["weight"] - base["weight"]))
        sp["unstable"] |= o2["status"] != base["status"]
        sp["tiles"].append(o2["tile_id"])
    return sp


def oracle_trace(cloak, integ, mode, rays):
    base = O.trace_rays(cloak, integ, mode, rays)
    others = [O.trace_rays(cloak, integ, mode, perturb_rays(rays, k)) for k in range(4)]
    return base, spread_of(base, others)


def tile_edge_gap(pos, d, H=2.0):
    """Distance (in units of length) from the room hit point to the nearest tile edge or
    face boundary, for the procedural room x, y in [-10, 10], z in [-H/2, -H/2 + 10]."""
    Lb, z0 = 10.0, -0.5 * H
    lo = np.array([-Lb, -Lb, z0])
    hi = np.array([Lb, Lb, z0 + 10.0])
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(d > 0, (hi - pos) / d, np.where(d < 0, (lo - pos) / d, np.inf))
    ss = np.sort(s, axis=1)
    q = pos + ss[:, :1] * d
    frac = lambda t: np.abs(t * 8 - np.round(t * 8)) / 8
    gap = np.minimum(frac(q[:, 0] + Lb), np.minimum(frac(q[:, 1] + Lb), frac(q[:, 2] - z0)))
    face_gap = (ss[:, 1] - ss[:, 0]) * np.abs(d).min(1)
    return np.minimum(gap + 0.0, np.where(np.isfinite(face_gap), face_gap, np.inf))


def compare_records(g, o, sp, what, steps_exact=True, max_unstable=0.02, H=2.0, noise_limited=None):
    """Element-by-element comparison of GPU and oracle records (see module docstring).  noise_limited:
    mask of rays whose time of flight FP64 does not fix at the tolerance (checked for validity only)."""
    assert g.shape == o.shape
    n = len(o)
    uns = sp["unstable"]
    assert uns.mean() <= max_unstable, f"{what}: {uns.sum()} of {n} rays change status under a 1e-13 perturbation"
    st = ~uns
    bad = np.nonzero(st & (g["status"] != o["status"]))[0]
    assert len(bad) == 0, f"{what}: {len(bad)} status mismatches, e.g. idx {bad[:5]} gpu {g['status'][bad[:5]]} " \
                          f"oracle {o['status'][bad[:5]]}"
    assert np.array_equal(g["mode"], o["mode"])
    # validity of the rays whose status FP64 does not determine
    assert np.isin(g["status"][uns], np.arange(8)).all()
    fin = np.isin(o["status"], [0, 1, 2, 7]) & st
    ang = angles(g["exit_dir"][fin], o["exit_dir"][fin])
    lim = TOL_DIR + KAPPA * sp["dir"][fin]
    over = np.nonzero(ang > lim)[0]
    assert len(over) == 0, f"{what}: exit direction off by {ang[over[:3]]} rad (allowed {lim[over[:3]]})"
    for key, field in (("pos", "exit_pos"), ("tof", "tof"), ("w", "weight")):
        sel = st & ~noise_limited if (key == "tof" and noise_limited is not None) else st
        dv = np.abs(g[field][sel] - o[field][sel])
        if dv.ndim > 1:
            dv = dv.max(1)
        lim2 = TOL_ABS + KAPPA * sp[key][sel]
        over = np.nonzero(dv > lim2)[0]
        assert len(over) == 0, f"{what}: {field} off by {dv[over[:3]]} (allowed {lim2[over[:3]]})"
    tb = np.nonzero(st & (g["tile_id"] != o["tile_id"]))[0]
    if len(tb):
        seen = np.stack(sp["tiles"], 1)[tb]
        tie = (tile_edge_gap(o["exit_pos"][tb], o["exit_dir"][tb], H) < 1e-9) | (seen == g["tile_id"][tb, None]).any(1)
        assert tie.all(), f"{what}: {(~tie).sum()} tile mismatches away from a tile edge"
    if steps_exact:
        sb = np.nonzero(st & (g["steps"] != o["steps"]) & (sp["dir"] < 1e-12))[0]
        assert len(sb) == 0, f"{what}: {len(sb)} step-count mismatches"
    wc = sp["dir"][fin] <= 0.1 * TOL_DIR
    return dict(max_dir_err=float(ang.max(initial=0)), max_dir_err_wellcond=float(ang[wc].max(initial=0)),
                illcond_frac=float(1 - wc.mean()) if len(wc) else 0.0, unstable=int(uns.sum()))


def gpu_trace(ck, variant, mode, rays, integ, h_or_tol, max_steps=1_000_000, test_medium=None, R1=0.5, R2=1.0,
              height=2.0):
    import torch
    c = ck.Cloak(variant, R1=R1, R2=R2, height=height)
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
    o, sp = oracle_trace(O.Cloak(variant), O.Integrator(integ, h_or_tol), mode, rays)
    stats = compare_records(g, o, sp, f"v{variant} m{mode} i{integ}", steps_exact=(integ == 0), max_unstable=0.05)
    print(stats)
    # the ray set reaches every branch the variant/mode allows
    assert (o["status"] == 0).sum() > 50 and np.isin(o["status"], [1, 2]).sum() > 300


@pytest.mark.parametrize("mode", [0, 1])
def test_test_medium_interfaces(ck, mode):
    """Homogeneous uniaxial cylinder with a tilted optic axis: entry and exit
    refraction (Sect. 3) and Eq. 12 weights for a general c-hat."""
    rays = inputs.ray_set(500, seed=5, kind="mixed")
    med = (2.2, 3.1, (0.5, -0.3, 0.81))
    g = gpu_trace(ck, 100, mode, rays, 0, 1e-2, test_medium=med, R1=0.0)
    o, sp = oracle_trace(O.Cloak(O.TEST_CONST, R1=0.0, eps_o=2.2, eps_e=3.1, c_hat=(0.5, -0.3, 0.81)),
                         O.Integrator(O.RK4, 1e-2), mode, rays)
    compare_records(g, o, sp, f"test medium m{mode}")
    assert np.isin(o["status"], [1]).sum() > 200


SCHEDULES = ("plain", "wavefront")


def small_render(ck, variant, mode, integ, h_or_tol, W, H, spp, elev, seed=0, records=True, schedule="plain",
                 precision=0, geom=(0.5, 1.0, 2.0)):
    """geom: (R1, R2, height) of the cloak."""
    import torch
    eye, tgt, up = inputs.camera_pose(elev)
    c = ck.Cloak(variant, *geom).camera(eye, tgt, up, 60.0, W, H).integrator(integ, h_or_tol, precision)
    c.schedule(ck.SCHED_WAVEFRONT if schedule == "wavefront" else ck.SCHED_PLAIN)
    img = c.render(mode, spp, seed)
    rec = c.render_records(mode, spp, seed) if records else None
    torch.cuda.synchronize()
    img = img.reshape(-1, 4).cpu().numpy().astype(np.float64)
    rec = ck.records_to_numpy(rec) if records else None
    c.close()
    return img, rec


def oracle_render(variant, mode, integ, h_or_tol, W, H, spp, elev, seed, pixels=None, geom=(0.5, 1.0, 2.0)):
    """Oracle image and records, plus the spread under 1e-13 perturbations of the camera."""
    eye, tgt, up = inputs.camera_pose(elev)
    integ_o = O.Integrator(integ, h_or_tol)
    cl = O.Cloak(variant, R1=geom[0], R2=geom[1], H=geom[2])
    rgba, rec = O.render(cl, integ_o, O.Camera(eye, tgt, up, 60, W, H), mode, spp, seed, pixels=pixels)
    others = []
    for k in range(3):
        rng = np.random.default_rng(2000 + k)
        e2 = np.array(eye) + PERTURB * rng.normal(size=3)
        t2 = np.array(tgt) + PERTURB * rng.normal(size=3)
        others.append(O.render(cl, integ_o, O.Camera(e2, t2, up, 60, W, H), mode, spp, seed,
                               pixels=pixels)[1])
    return rgba, rec, spread_of(rec, others)


def compare_images(img, rgba, rec, orec, sp, spp, what):
    """RGBA within 1e-5 wherever every sample of the pixel has a determined status and tile."""
    good = (~sp["unstable"]) & (rec["tile_id"] == orec["tile_id"]) & (sp["dir"] <= 0.1 * TOL_DIR)
    good = good.reshape(-1, spp).all(1)
    assert np.all(np.isfinite(img)) and img.min() >= 0.0 and img.max() <= 1.0 + 1e-6
    d = np.abs(img[good] - rgba[good]).max(initial=0)
    assert d < 1e-5, f"{what}: RGBA differs by {d}"
    return float(1 - good.mean())


def test_small_config_image(ck):
    """The small workload (radial, extraordinary, 128x96, 1 spp, RK4 h = 1e-3): whole image."""
    w = inputs.SMALL
    rgba, orec, sp = oracle_render(0, 1, 0, 1e-3, w.width, w.height, 1, 0.0, 0)
    for sched in SCHEDULES:
        img, rec = small_render(ck, 0, 1, 0, 1e-3, w.width, w.height, 1, 0.0, schedule=sched)
        stats = compare_records(rec, orec, sp, f"small image {sched}")
        frac = compare_images(img, rgba, rec, orec, sp, 1, f"small image {sched}")
        print(sched, stats, "pixels without a determined tile:", frac)
        assert frac < 0.002
    assert (orec["status"] == 1).sum() > 1500


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_jittered_elevations_dp45(ck, variant, mode):
    """Both variants and polarizations, elevations 0/20/45 deg, 2 jittered samples,
    DP5(4) at tol 1e-9, 61x37 pixels (a ragged tail for 128-thread blocks)."""
    W, H, spp = 61, 37, 2
    for elev in (0.0, 20.0, 45.0):
        rgba, orec, sp = oracle_render(variant, mode, 1, 1e-9, W, H, spp, elev, 3)
        for sched in SCHEDULES:
            img, rec = small_render(ck, variant, mode, 1, 1e-9, W, H, spp, elev, seed=3, schedule=sched)
            stats = compare_records(rec, orec, sp, f"v{variant} m{mode} e{elev} {sched}", steps_exact=False)
            compare_images(img, rgba, rec, orec, sp, spp, f"v{variant} m{mode} e{elev} {sched}")
            print(elev, sched, stats)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_full_size_sampled(ck, schedule):
    """1920x1080, 4 jittered spp, DP5(4) tol 1e-9 (the full workload's launch shape),
    azimuthal cloak, extraordinary light, elevation 20 deg: a seeded sample of pixels
    against the oracle; validity over every pixel."""
    import torch
    w = inputs.FULL
    eye, tgt, up = inputs.camera_pose(20.0)
    c = ck.Cloak(1).camera(eye, tgt, up, 60.0, w.width, w.height).integrator(1, 1e-9)
    c.schedule(ck.SCHED_WAVEFRONT if schedule == "wavefront" else ck.SCHED_PLAIN)
    rec_t = c.render_records(1, w.spp, w.seed)
    img = c.render(1, w.spp, w.seed)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    pix = np.sort(rng.choice(w.width * w.height, 400, replace=False))
    rec = ck.records_to_numpy(rec_t).reshape(-1, w.spp)[pix].reshape(-1)
    rgba_g = img.reshape(-1, 4).cpu().numpy().astype(np.float64)
    rgba, orec, sp = oracle_render(1, 1, 1, 1e-9, w.width, w.height, w.spp, 20.0, w.seed, pixels=pix)
    stats = compare_records(rec, orec, sp, "full-size sample", steps_exact=False)
    compare_images(rgba_g[pix], rgba, rec, orec, sp, w.spp, "full-size sample")
    print(stats)
    allrec = ck.records_to_numpy(rec_t)
    assert np.all(np.isfinite(rgba_g))
    assert np.isin(allrec["status"], [0, 1, 2, 3, 4, 5, 6, 7]).all()
    assert (allrec["status"] == 5).mean() < 1e-4
    c.close()


def test_edge_cases(ck):
    import torch
    c = ck.Cloak(0)
    # empty ray batch
    out = torch.empty(80, dtype=torch.uint8, device="cuda")
    ck.cloak_trace_rays(c.h, 1, torch.empty((0, 6), dtype=torch.float64, device="cuda"), 0, out)
    # 1x1 and odd images
    for W, H, spp in ((1, 1, 1), (7, 5, 3)):
        rgba, orec, sp = oracle_render(0, 1, 0, 1e-3, W, H, spp, 0.0, 9)
        for sched in SCHEDULES:
            img, rec = small_render(ck, 0, 1, 0, 1e-3, W, H, spp, 0.0, seed=9, schedule=sched)
            # the single pixel of a 1x1 image looks exactly along the axis (impact parameter 0)
            compare_records(rec, orec, sp, f"{W}x{H} {sched}", max_unstable=1.0)
            compare_images(img, rgba, rec, orec, sp, spp, f"{W}x{H} {sched}")
    # step limit
    rays = inputs.ray_set(64, seed=2, kind="lateral")
    g = gpu_trace(ck, 1, 1, rays, 0, 1e-3, max_steps=7)
    o, sp = oracle_trace(O.Cloak(1), O.Integrator(0, 1e-3, 7), 1, rays)
    assert (o["status"] == 5).sum() > 30
    compare_records(g, o, sp, "max_steps=7")
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


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_wavefront_matches_plain(ck, variant, mode):
    """Both schedules run the same per-ray arithmetic (up to the compiler's FMA contraction in
    different inlining contexts): statuses and tiles agree exactly, exit directions within the
    FP64 bar (here at 320x180, 4 spp, DP5(4), elevation 20 deg, and RK4 at elevation 45 deg)."""
    for integ, tol, elev in ((1, 1e-9, 20.0), (0, 1e-3, 45.0)):
        a_img, a_rec = small_render(ck, variant, mode, integ, tol, 320, 180, 4, elev, seed=5, schedule="plain")
        b_img, b_rec = small_render(ck, variant, mode, integ, tol, 320, 180, 4, elev, seed=5, schedule="wavefront")
        assert np.array_equal(a_rec["status"], b_rec["status"])
        assert np.array_equal(a_rec["tile_id"], b_rec["tile_id"])
        assert angles(a_rec["exit_dir"], b_rec["exit_dir"]).max() < TOL_DIR
        assert np.abs(a_rec["tof"] - b_rec["tof"]).max() < TOL_ABS
        assert np.abs(a_img - b_img).max() < 1e-6


# Cloak shapes away from R1 = 0.5, R2 = 1, height 2: a thin core (K = 1.11, nearly vacuum), a thin shell
# (K = 100: strong anisotropy, rays that crawl around the metal) and a squat cloak of another scale
# (nothing in the kernels may assume R2 = 1 or a fixed height).
GEOMETRIES = ((0.05, 1.0, 2.0), (0.9, 1.0, 2.0), (1.2, 3.0, 0.7))


@pytest.mark.parametrize("geom", GEOMETRIES)
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_geometry_trace_rays_parity(ck, geom, variant, mode):
    """Ray sets scaled to each cloak shape, DP5(4) tol 1e-9, FP64 bar.

    In the thin shell, near-axis extraordinary rays of the azimuthal cloak crawl within 1.5e-5 of R1
    (1/f ~ 4e7 there).  Their step attempts grow 10x per decade of tolerance instead of the 1.6x of a
    fifth-order method: the embedded error estimate is rounding noise, and the step sequences of two
    FP64 programs part ways.  For these rays (steps at tol 1e-9 over 5x those at 1e-8) the time of
    flight, which the oracle itself moves by ~4e-5 between tolerances 1e-8, 1e-9 and 1e-10, is checked
    for validity only; status, exit direction, exit point and weight keep the FP64 bar.  Up to ~1e6
    step attempts, so the limit is 2e6."""
    R1, R2, H = geom
    rays = inputs.ray_set(240, seed=31 + 2 * variant + mode, kind="mixed", R2=R2, H=H, distance=3.0 * R2)
    g = gpu_trace(ck, variant, mode, rays, 1, 1e-9, max_steps=2_000_000, R1=R1, R2=R2, height=H)
    cl = O.Cloak(variant, R1=R1, R2=R2, H=H)
    o, sp = oracle_trace(cl, O.Integrator(1, 1e-9, 2_000_000), mode, rays)
    assert (o["status"] != 5).all()
    coarse = O.trace_rays(cl, O.Integrator(1, 1e-8, 2_000_000), mode, rays)
    noisy = o["steps"] > 5 * np.maximum(coarse["steps"], 1)
    assert noisy.mean() <= 0.1
    assert np.all(np.isfinite(g["tof"][noisy]) & (g["tof"][noisy] > 0))
    stats = compare_records(g, o, sp, f"R1={R1} R2={R2} H={H} v{variant} m{mode}", steps_exact=False,
                            max_unstable=0.05, H=H, noise_limited=noisy)
    stats["noise_limited"] = int(noisy.sum())
    print(stats)
    assert np.isin(o["status"], [1, 2]).sum() > 100


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_geometry_render_wavefront(ck, variant, mode):
    """Camera renders of the squat cloak of radius 3 through the wavefront schedule, FP64 DP5(4)."""
    geom = (1.2, 3.0, 0.7)
    W, H, spp = 64, 48, 2
    rgba, orec, sp = oracle_render(variant, mode, 1, 1e-9, W, H, spp, 20.0, 3, geom=geom)
    img, rec = small_render(ck, variant, mode, 1, 1e-9, W, H, spp, 20.0, seed=3, schedule="wavefront", geom=geom)
    compare_records(rec, orec, sp, f"squat cloak v{variant} m{mode}", steps_exact=False, H=geom[2])
    compare_images(img, rgba, rec, orec, sp, spp, f"squat cloak v{variant} m{mode}")
    assert np.isin(orec["status"], [1, 2]).mean() > 0.2
