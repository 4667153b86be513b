"""GPU-vs-oracle parity of the FP64 path (through the C ABI).

Bar (FP64): exit directions within 1e-9 rad of the oracle, exit points, times of flight and Eq. 12
weights within 1e-9, statuses identical, RK4 step counts identical, room tiles identical (a mismatch is
accepted only where the oracle's hit point lies on a tile edge); images (FP32 colour accumulation) within
1e-5.

The reference is the oracle.  Where the FP64 oracle does not determine a ray -- it disagrees with the same
source in long double by more than 1e-10 (status, exit direction, point, time of flight or weight): near
r = R1 the literal Cartesian form of Eq. 8 loses digits to cancellation -- the reference is that oracle
source in IEEE binary128 at the same step or tolerance (tests/golden/parity/, written by
make_parity_references.py).  Those rays keep the 1e-9 bars, widened only by 8 x D64, where D64 is how far
the binary128 run moves when its states and stage points are rounded to FP64 (what FP64 can determine at
best).  The exit direction, exit point and time of flight share the largest of their three D64: one
displacement of the path shows in all three, and a single perturbed run can leave one of them small by
chance (on a near-axis ray of the full workload the GPU's time of flight moved 40 times its own D64, 5 times
the shared one).  The weight keeps its own D64.
"""
import os

import numpy as np
import pytest

import oracle as O
import parity_cases as P
from paper_1209_6038_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_DIR = 1e-9      # FP64 exit-direction bar (rad)
TOL_ABS = 1e-9      # exit point, time of flight, weight
D64_FACTOR = 8.0    # multiple of D64 added to the bar of a ray the FP64 oracle does not determine
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "parity")


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


def reference(name, spec=None):
    """Records of parity case `name` from the FP64 oracle, with the binary128 reference in place of every
    ray the FP64 oracle does not determine; returns (records, per-ray bars, undetermined mask).  The bars:
    a dict of per-ray arrays for the exit direction ("dir", rad) and for "exit_pos", "tof" and "weight"."""
    ref = P.oracle_records(O, spec or P.cases()[name]).copy()
    lim = {k: np.full(len(ref), TOL_DIR if k == "dir" else TOL_ABS) for k in ("dir", "exit_pos", "tof", "weight")}
    und = np.zeros(len(ref), bool)
    for line in open(os.path.join(GOLDEN, name + ".txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        k = int(f[0])
        ref["status"][k], ref["steps"][k] = int(f[1]), int(f[2])
        ref["exit_dir"][k] = [float(x) for x in f[3:6]]
        ref["exit_pos"][k] = [float(x) for x in f[6:9]]
        ref["tof"][k], ref["weight"][k], ref["tile_id"][k] = float(f[9]), float(f[10]), int(f[11])
        d64 = [float(x) for x in f[12:16]]
        for key in ("dir", "exit_pos", "tof"):
            lim[key][k] += D64_FACTOR * max(d64[:3])
        lim["weight"][k] += D64_FACTOR * d64[3]
        und[k] = True
    return ref, lim, und


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


def compare_records(g, ref, lim, und, what, steps_exact=True, H=2.0):
    """Element-by-element comparison of GPU records with the reference (see the module docstring)."""
    assert g.shape == ref.shape
    bad = np.nonzero(g["status"] != ref["status"])[0]
    assert len(bad) == 0, f"{what}: {len(bad)} status mismatches, e.g. idx {bad[:5]} gpu {g['status'][bad[:5]]} " \
                          f"reference {ref['status'][bad[:5]]}"
    assert np.array_equal(g["mode"], ref["mode"])
    fin = np.isin(ref["status"], [0, 1, 2, 7])
    ang = angles(g["exit_dir"][fin], ref["exit_dir"][fin])
    over = np.nonzero(ang > lim["dir"][fin])[0]
    assert len(over) == 0, f"{what}: exit direction off by {ang[over[:3]]} rad (allowed {lim['dir'][fin][over[:3]]}) " \
                           f"at rays {np.nonzero(fin)[0][over[:3]]}"
    for field in ("exit_pos", "tof", "weight"):
        dv = np.abs(g[field] - ref[field])
        if dv.ndim > 1:
            dv = dv.max(1)
        over = np.nonzero(dv > lim[field])[0]
        assert len(over) == 0, f"{what}: {field} off by {dv[over[:3]]} (allowed {lim[field][over[:3]]}) at rays {over[:3]}"
    tb = np.nonzero(g["tile_id"] != ref["tile_id"])[0]
    if len(tb):
        tie = tile_edge_gap(ref["exit_pos"][tb], ref["exit_dir"][tb], H) < 1e-9
        assert tie.all(), f"{what}: {(~tie).sum()} tile mismatches away from a tile edge"
    if steps_exact:
        sb = np.nonzero((g["steps"] != ref["steps"]) & ~und)[0]
        assert len(sb) == 0, f"{what}: {len(sb)} step-count mismatches"
    return dict(max_dir_err=float(ang.max(initial=0)),
                max_dir_err_determined=float(ang[~und[fin]].max(initial=0)),
                undetermined=int(und.sum()), widened=int((lim["dir"] > TOL_DIR).sum()), rays=len(ref))


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


def gpu_case(ck, spec):
    """GPU records of a ray-set case."""
    s = P.materialise(spec)
    R1, R2, H = s["geometry"]
    return gpu_trace(ck, s["variant"], s["mode"], s["rays"], s["integ"], s["h_or_tol"], s["max_steps"],
                     test_medium=s.get("medium"), R1=R1, R2=R2, height=H)


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("integ", [0, 1])
def test_trace_rays_parity(ck, variant, mode, integ):
    name = f"rays_v{variant}_m{mode}_i{integ}"
    spec = P.cases()[name]
    g = gpu_case(ck, spec)
    ref, lim, und = reference(name)
    stats = compare_records(g, ref, lim, und, name, steps_exact=(integ == 0))
    print(stats)
    # the ray set reaches every branch the variant/mode allows
    assert (ref["status"] == 0).sum() > 50 and np.isin(ref["status"], [1, 2]).sum() > 300


@pytest.mark.parametrize("mode", [0, 1])
def test_test_medium_interfaces(ck, mode):
    """Homogeneous uniaxial cylinder with a tilted optic axis: entry and exit
    refraction (Sect. 3) and Eq. 12 weights for a general c-hat."""
    name = f"test_medium_m{mode}"
    g = gpu_case(ck, P.cases()[name])
    ref, lim, und = reference(name)
    compare_records(g, ref, lim, und, name)
    assert np.isin(ref["status"], [1]).sum() > 200


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


def render_case(ck, name, schedule):
    s = P.materialise(P.cases()[name])
    return small_render(ck, s["variant"], s["mode"], s["integ"], s["h_or_tol"], s["width"], s["height"], s["spp"],
                        s["elevation"], seed=s["seed"], schedule=schedule, geom=s["geometry"])


def oracle_image(name):
    """The oracle's RGBA of a render case (FP64)."""
    s = P.materialise(P.cases()[name])
    R1, R2, H = s["geometry"]
    eye, tgt, up = inputs.camera_pose(s["elevation"])
    return O.render(O.Cloak(s["variant"], R1=R1, R2=R2, H=H), O.Integrator(s["integ"], s["h_or_tol"]),
                    O.Camera(eye, tgt, up, 60.0, s["width"], s["height"]), s["mode"], s["spp"], s["seed"],
                    pixels=s["pixels"], records=False)[0]


def compare_images(img, rgba, rec, ref, und, spp, what):
    """RGBA within 1e-5 wherever every sample of the pixel is determined by the FP64 oracle and sees the
    reference's tile."""
    good = (~und) & (rec["tile_id"] == ref["tile_id"])
    good = good.reshape(-1, spp).all(1)
    assert np.all(np.isfinite(img)) and img.min() >= 0.0 and img.max() <= 1.0 + 1e-6
    d = np.abs(img[good] - rgba[good]).max(initial=0)
    assert d < 1e-5, f"{what}: RGBA differs by {d}"
    return float(1 - good.mean())


def test_small_config_image(ck):
    """The small workload (radial, extraordinary, 128x96, 1 spp, RK4 h = 1e-3): whole image."""
    ref, lim, und = reference("render_small")
    rgba = oracle_image("render_small")
    for sched in SCHEDULES:
        img, rec = render_case(ck, "render_small", sched)
        stats = compare_records(rec, ref, lim, und, f"small image {sched}")
        frac = compare_images(img, rgba, rec, ref, und, 1, f"small image {sched}")
        print(sched, stats, "pixels not compared:", frac)
        assert frac < 0.002
    assert (ref["status"] == 1).sum() > 1500


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_jittered_elevations_dp45(ck, variant, mode):
    """Both variants and polarizations, elevations 0/20/45 deg, 2 jittered samples,
    DP5(4) at tol 1e-9, 61x37 pixels (a ragged tail for 128-thread blocks)."""
    for elev in (0, 20, 45):
        name = f"render_jitter_v{variant}_m{mode}_e{elev}"
        ref, lim, und = reference(name)
        rgba = oracle_image(name)
        for sched in SCHEDULES:
            img, rec = render_case(ck, name, sched)
            stats = compare_records(rec, ref, lim, und, f"{name} {sched}", steps_exact=False)
            compare_images(img, rgba, rec, ref, und, 2, f"{name} {sched}")
            print(elev, sched, stats)


@pytest.mark.parametrize("schedule", SCHEDULES)
def test_full_size_sampled(ck, schedule):
    """1920x1080, 4 jittered spp, DP5(4) tol 1e-9 (the full workload's launch shape),
    azimuthal cloak, extraordinary light, elevation 20 deg: a seeded sample of pixels
    against the oracle; validity over every pixel."""
    import torch
    name = "render_full_sampled"
    s = P.materialise(P.cases()[name])
    w = inputs.FULL
    eye, tgt, up = inputs.camera_pose(20.0)
    c = ck.Cloak(1).camera(eye, tgt, up, 60.0, w.width, w.height).integrator(1, 1e-9)
    c.schedule(ck.SCHED_WAVEFRONT if schedule == "wavefront" else ck.SCHED_PLAIN)
    rec_t = c.render_records(1, w.spp, w.seed)
    img = c.render(1, w.spp, w.seed)
    torch.cuda.synchronize()
    pix = s["pixels"]
    rec = ck.records_to_numpy(rec_t).reshape(-1, w.spp)[pix].reshape(-1)
    rgba_g = img.reshape(-1, 4).cpu().numpy().astype(np.float64)
    ref, lim, und = reference(name, s)
    rgba = oracle_image(name)
    stats = compare_records(rec, ref, lim, und, "full-size sample", steps_exact=False)
    compare_images(rgba_g[pix], rgba, rec, ref, und, w.spp, "full-size sample")
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
    # 1x1 and odd images; the single pixel of a 1x1 image looks exactly along the axis (impact parameter 0:
    # the extraordinary ray of the radial cloak reaches r = R1, status SINGULAR)
    for W, H, spp in ((1, 1, 1), (7, 5, 3)):
        name = f"render_edge_{W}x{H}x{spp}"
        ref, lim, und = reference(name)
        rgba = oracle_image(name)
        for sched in SCHEDULES:
            img, rec = render_case(ck, name, sched)
            compare_records(rec, ref, lim, und, f"{W}x{H} {sched}")
            compare_images(img, rgba, rec, ref, und, spp, f"{W}x{H} {sched}")
    # step limit
    g = gpu_case(ck, P.cases()["rays_step_limit"])
    ref, lim, und = reference("rays_step_limit")
    assert (ref["status"] == 5).sum() > 30
    compare_records(g, ref, lim, und, "max_steps=7")
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


@pytest.mark.parametrize("geom", P.GEOMETRIES)
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_geometry_trace_rays_parity(ck, geom, variant, mode):
    """Cloak shapes away from R1 = 0.5, R2 = 1, height 2: a thin core (K = 1.11, nearly vacuum), a thin
    shell (K = 100: strong anisotropy, rays that crawl around the metal) and a squat cloak of another
    scale (nothing in the kernels may assume R2 = 1 or a fixed height).  Ray sets scaled to each shape,
    DP5(4) tol 1e-9, up to 2e6 step attempts, FP64 bar."""
    name = f"geom_{P._geom_name(geom)}_v{variant}_m{mode}"
    g = gpu_case(ck, P.cases()[name])
    ref, lim, und = reference(name)
    stats = compare_records(g, ref, lim, und, name, steps_exact=False, H=geom[2])
    print(stats)
    assert (ref["status"] != 5).all()
    assert np.isin(ref["status"], [1, 2]).sum() > 100


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_geometry_render_wavefront(ck, variant, mode):
    """Camera renders of the squat cloak of radius 3 through the wavefront schedule, FP64 DP5(4)."""
    name = f"render_squat_v{variant}_m{mode}"
    ref, lim, und = reference(name)
    rgba = oracle_image(name)
    img, rec = render_case(ck, name, "wavefront")
    compare_records(rec, ref, lim, und, name, steps_exact=False, H=0.7)
    compare_images(img, rgba, rec, ref, und, 2, name)
    assert np.isin(ref["status"], [1, 2]).mean() > 0.2
