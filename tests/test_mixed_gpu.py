"""Mixed-precision path (FP32 right-hand sides and stage combinations, float-float state,
FP64 or double-float steps within 0.02 of the inner radius, FP64 interface solves) against the FP64 oracle.

Bar: exit direction within 1e-5 rad of the oracle, and at least 99.9% of sampled pixels with the
same room tile and status in every sample.  As in the FP64 tests the bar widens where the problem
itself amplifies rounding: the oracle's own change under 1e-13 input perturbations (its spread),
scaled to FP32 rounding (2^-24 / 1e-13), times 10, is added per ray -- e.g. near-grazing exits
through a cap, where the exit direction is 1/sqrt(1 - |k_t|^2) times more sensitive than k.
"""
import numpy as np
import pytest

import oracle as O
from paper_1209_6038_gb300 import inputs
from test_parity_gpu import PERTURB, angles, ck, oracle_render, small_render  # noqa: F401

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-5
FP32_OVER_PROBE = 2.0 ** -24 / PERTURB


def mixed_errors(rec, orec, sp):
    same = rec["status"] == orec["status"]
    fin = same & np.isin(orec["status"], [0, 1, 2, 7]) & ~sp["unstable"]
    err = angles(rec["exit_dir"][fin], orec["exit_dir"][fin])
    lim = TOL_MIXED + 10 * FP32_OVER_PROBE * sp["dir"][fin]
    return err, lim, same


# the band near R1 in FP64 (CLOAK_MIXED) or in double-float (CLOAK_MIXED_FF)
BANDS = [1, 2]


@pytest.mark.parametrize("band", BANDS)
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_mixed_exit_directions(ck, variant, mode, band):
    W, H, spp = 96, 54, 2
    worst = 0.0
    for elev in (0.0, 20.0, 45.0):
        rgba, orec, sp = oracle_render(variant, mode, 1, 1e-9, W, H, spp, elev, 7)
        img, rec = small_render(ck, variant, mode, 1, 1e-9, W, H, spp, elev, seed=7, schedule="wavefront",
                                precision=band)
        err, lim, same = mixed_errors(rec, orec, sp)
        over = np.nonzero(err > lim)[0]
        assert len(over) == 0, f"v{variant} m{mode} e{elev}: exit-direction errors {err[over[:5]]}"
        assert (~same).mean() < 0.005, f"v{variant} m{mode} e{elev}: {(~same).sum()} status changes"
        worst = max(worst, float(err.max(initial=0)))
        assert np.all(np.isfinite(img))
    print(f"v{variant} m{mode}: max exit-direction error {worst:.2e} rad")


@pytest.mark.parametrize("band", BANDS)
def test_mixed_rk4_small_config(ck, band):
    """The small workload (radial, extraordinary, RK4 h = 1e-3) on the mixed path."""
    w = inputs.SMALL
    rgba, orec, sp = oracle_render(0, 1, 0, 1e-3, w.width, w.height, 1, 0.0, 0)
    img, rec = small_render(ck, 0, 1, 0, 1e-3, w.width, w.height, 1, 0.0, schedule="wavefront", precision=band)
    err, lim, same = mixed_errors(rec, orec, sp)
    assert np.all(err <= lim)
    assert (~same).mean() < 0.005


@pytest.mark.parametrize("band", BANDS)
def test_mixed_full_size_pixels(ck, band):
    """1920x1080, 4 spp, DP5(4) tol 1e-9, azimuthal e-light at 20 deg: >= 99.9% of 2000 sampled
    pixels keep every sample's tile and status."""
    import torch
    w = inputs.FULL
    eye, tgt, up = inputs.camera_pose(20.0)
    c = ck.Cloak(1).camera(eye, tgt, up, 60.0, w.width, w.height).integrator(1, 1e-9, band)
    c.schedule(ck.SCHED_WAVEFRONT)
    rec_t = c.render_records(1, w.spp, w.seed)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    pix = np.sort(rng.choice(w.width * w.height, 2000, replace=False))
    rec = ck.records_to_numpy(rec_t).reshape(-1, w.spp)[pix].reshape(-1)
    c.close()
    _, orec = O.render(O.Cloak(1), O.Integrator(1, 1e-9), O.Camera(eye, tgt, up, 60, w.width, w.height), 1, w.spp,
                       w.seed, pixels=pix)
    diff = ((rec["tile_id"] != orec["tile_id"]) | (rec["status"] != orec["status"])).reshape(-1, w.spp).any(1)
    assert diff.mean() <= 1e-3, f"{diff.sum()} of {len(pix)} pixels differ"
    fin = (rec["status"] == orec["status"]) & np.isin(orec["status"], [0, 1, 2, 7])
    err = angles(rec["exit_dir"][fin], orec["exit_dir"][fin])
    print("full-size mixed: max exit-direction error", err.max(), "differing pixels", diff.sum())
    assert np.quantile(err, 0.999) <= TOL_MIXED


def test_mixed_needs_wavefront(ck):
    import torch
    c = ck.Cloak(0).integrator(1, 1e-9, ck.MIXED)
    with pytest.raises(ck.CloakError):
        c.render(1, 1, 0)
    c.close()


@pytest.mark.parametrize("band", BANDS)
@pytest.mark.parametrize("geom", [(0.9, 1.0, 2.0), (1.2, 3.0, 0.7)])
@pytest.mark.parametrize("variant", [0, 1])
def test_mixed_other_geometries(ck, geom, variant, band):
    """The mixed path on a thin shell (K = 100) and on a squat cloak of radius 3, extraordinary light."""
    W, H, spp = 64, 48, 2
    rgba, orec, sp = oracle_render(variant, 1, 1, 1e-9, W, H, spp, 20.0, 4, geom=geom)
    img, rec = small_render(ck, variant, 1, 1, 1e-9, W, H, spp, 20.0, seed=4, schedule="wavefront", precision=band,
                            geom=geom)
    err, lim, same = mixed_errors(rec, orec, sp)
    over = np.nonzero(err > lim)[0]
    assert len(over) == 0, f"{geom} v{variant}: exit-direction errors {err[over[:5]]}"
    assert (~same).mean() < 0.005, f"{geom} v{variant}: {(~same).sum()} status changes"
    assert np.all(np.isfinite(img))
    print(f"{geom} v{variant}: max exit-direction error {err.max(initial=0):.2e} rad")
