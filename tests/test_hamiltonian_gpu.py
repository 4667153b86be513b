"""The Hamiltonian form of the ray equations on the GPU against the oracle's Hamiltonian traces (same
integrator, crossings and interfaces), on the plain and wavefront schedules; and its agreement with the
Fermat form (both converge to the same rays)."""
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


def exit_angle(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("variant,mode", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_hamiltonian_records_match_the_oracle(ck, schedule, variant, mode):
    W, H = 48, 32
    eye, tgt, up = inputs.camera_pose(20.0, 5.0)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, ck.FP64, 1_000_000)
    c.schedule(schedule).formulation(ck.FORM_HAMILTONIAN)
    g = ck.records_to_numpy(c.render_records(mode))
    _, o = O.render(O.Cloak(variant, form=O.HAMILTONIAN), O.Integrator(O.DP45, 1e-9, 1_000_000),
                    O.Camera(eye, tgt, up, 60.0, W, H), mode, spp=1, seed=0)
    same = g["status"] == o["status"]
    assert same.mean() > 0.99
    fin = same & np.isin(o["status"], [1, 2])
    L = np.abs(o["exit_pos"][:, 0] * o["exit_dir"][:, 1] - o["exit_pos"][:, 1] * o["exit_dir"][:, 0])
    well = fin & (L > 1e-3)  # near-axis rays are ill-conditioned in any FP64 execution
    assert well.sum() > 20
    assert exit_angle(g["exit_dir"][well], o["exit_dir"][well]).max() < 1e-9
    assert np.max(np.abs(g["exit_pos"][well] - o["exit_pos"][well])) < 1e-9
    assert np.max(np.abs(g["weight"][well] - o["weight"][well])) < 1e-9
    assert np.array_equal(g["steps"][well], o["steps"][well]) or np.mean(g["steps"][well] == o["steps"][well]) > 0.98
    c.close()


def test_hamiltonian_and_fermat_forms_agree(ck):
    W, H = 64, 48
    eye, tgt, up = inputs.camera_pose(10.0)
    for variant in (0, 1):
        for mode in (0, 1):
            recs = []
            for form in (ck.FORM_FERMAT, ck.FORM_HAMILTONIAN):
                c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-11, ck.FP64)
                c.schedule(ck.SCHED_WAVEFRONT).formulation(form)
                recs.append(ck.records_to_numpy(c.render_records(mode)))
                c.close()
            a, b = recs
            fin = np.isin(a["status"], [1, 2]) & (a["status"] == b["status"])
            L = np.abs(a["exit_pos"][:, 0] * a["exit_dir"][:, 1] - a["exit_pos"][:, 1] * a["exit_dir"][:, 0])
            well = fin & (L > 1e-3)
            assert exit_angle(a["exit_dir"][well], b["exit_dir"][well]).max() < 1e-7


def test_formulation_needs_fp64_and_a_cloak(ck):
    c = ck.Cloak(0).integrator(ck.DP45, 1e-9, ck.MIXED)
    with pytest.raises(ck.CloakError):
        c.formulation(ck.FORM_HAMILTONIAN)
    c.integrator(ck.DP45, 1e-9, ck.FP64).formulation(ck.FORM_HAMILTONIAN)
    with pytest.raises(ck.CloakError):
        c.integrator(ck.DP45, 1e-9, ck.MIXED)
    c.close()
    t = ck.Cloak(ck.TEST_UNIAXIAL_CONST, R1=0.0)
    with pytest.raises(ck.CloakError):
        t.formulation(ck.FORM_HAMILTONIAN)
    t.close()


def test_hamiltonian_batch_matches_single_renders(ck):
    """The batched persistent form integrates the Hamiltonian form too: each view equals its own render."""
    import torch
    views, refs = [], []
    for variant, pol, elev, W, H in ((0, 1, 20.0, 64, 40), (1, 0, 0.0, 48, 48), (1, 1, 45.0, 56, 30)):
        eye, tgt, up = inputs.camera_pose(elev, 5.0)
        c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, ck.FP64)
        c.schedule(ck.SCHED_WAVEFRONT).formulation(ck.FORM_HAMILTONIAN)
        refs.append(c.render(pol, 2, 9).cpu().numpy())
        c.close()
        views.append((variant, pol, eye, tgt, up, 60.0, torch.empty((H, W, 4), device="cuda")))
    b = ck.Cloak(0).integrator(ck.DP45, 1e-9, ck.FP64).schedule(ck.SCHED_WAVEFRONT).formulation(ck.FORM_HAMILTONIAN)
    ck.cloak_render_batch(b.h, views, 2, 9)
    torch.cuda.synchronize()
    b.close()
    for (_, _, _, _, _, _, out), ref in zip(views, refs):
        assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-6
