"""Pins of the Hamiltonian form of the ray equations (the comparison system of Sect. 4's closing remark)
in the oracle: at k = M v it reproduces Eq. 8 (e) and Eq. 2 (o) -- dx/dt = v and dk/dt = d(M v)/dt along
the Fermat-form motion -- and RK4 in this form keeps H = (k^T M^-1 k - 1)/2 at zero to its truncation."""
import math

import numpy as np
import pytest

import oracle as O


def eps_o(cl, x):
    _, eo, _, _ = O.permittivity(cl, x)
    return eo


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
@pytest.mark.parametrize("mode", [O.ORDINARY, O.EXTRAORDINARY])
def test_hamiltonian_form_reproduces_the_fermat_form(variant, mode):
    cl = O.Cloak(variant)
    rng = np.random.default_rng(7 + variant + 2 * mode)
    for _ in range(25):
        r, ph, z = rng.uniform(0.55, 0.98), rng.uniform(0, 2 * math.pi), rng.uniform(-0.9, 0.9)
        x = np.array([r * math.cos(ph), r * math.sin(ph), z])
        v = rng.normal(0, 0.4, 3)
        if mode == O.EXTRAORDINARY:
            M, dM = O.aux_matrix(cl, x)
            M = M.reshape(3, 3)
            dM = dM.reshape(3, 3, 3)  # dM[k] = dM / dx_k
        else:
            eo = eps_o(cl, x)
            M = eo * np.eye(3)
            h = 1e-6
            dM = np.zeros((3, 3, 3))
            for kx in range(3):
                e1 = np.array(x)
                e2 = np.array(x)
                e1[kx] += h
                e2[kx] -= h
                dM[kx] = (eps_o(cl, e1) - eps_o(cl, e2)) / (2 * h) * np.eye(3)
        k = M @ v
        dyh = O.rhs_hamiltonian(cl, mode, np.concatenate([x, k]))
        dyf = O.rhs(cl, mode, np.concatenate([x, v]))
        # dx/dt = v
        assert np.max(np.abs(dyh[:3] - v)) < 1e-12 * max(1.0, np.abs(v).max())
        # dk/dt = d(M v)/dt = sum_l v_l (d_l M) v + M dv/dt
        dk = sum(v[l] * dM[l] @ v for l in range(3)) + M @ dyf[3:]
        tol = 1e-6 if mode == O.ORDINARY else 1e-11  # the ordinary gradient above is a central difference
        assert np.max(np.abs(dyh[3:] - dk)) < tol * max(1.0, np.abs(dk).max())


def test_rk4_in_hamiltonian_form_keeps_h_zero():
    cl = O.Cloak(O.AZIMUTHAL)
    x = np.array([0.9, 0.1, 0.0])
    # an extraordinary wave vector on the surface H = 0: scale a direction onto k^T M^-1 k = 1
    kd = np.array([-0.8, 0.5, 0.3])
    Mi = O.aux_inverse(cl, x).reshape(3, 3)
    k = kd / math.sqrt(kd @ Mi @ kd)
    y = np.concatenate([x, k])

    def H(y):
        Mi = O.aux_inverse(cl, y[:3]).reshape(3, 3)
        return 0.5 * (y[3:] @ Mi @ y[3:] - 1.0)

    def f(y):
        return O.rhs_hamiltonian(cl, O.EXTRAORDINARY, y)

    drift = {}
    for h in (4e-3, 2e-3):
        yy = y.copy()
        for _ in range(int(round(0.2 / h))):
            k1 = f(yy); k2 = f(yy + 0.5 * h * k1); k3 = f(yy + 0.5 * h * k2); k4 = f(yy + h * k3)
            yy = yy + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            assert math.hypot(yy[0], yy[1]) > 0.5
        drift[h] = abs(H(yy))
    assert drift[2e-3] < 1e-9 and drift[4e-3] / max(drift[2e-3], 1e-300) > 8  # fourth order


def test_hamiltonian_trace_agrees_with_the_fermat_trace():
    """Both forms integrate the same rays: their exits agree to the integrators' accuracy."""
    integ = O.Integrator(O.DP45, 1e-11, 2_000_000)
    rng = np.random.default_rng(11)
    n = 0
    for variant in (O.RADIAL, O.AZIMUTHAL):
        for mode in (O.ORDINARY, O.EXTRAORDINARY):
            for _ in range(6):
                o = np.array([4.0, rng.uniform(-0.9, 0.9), rng.uniform(-0.6, 0.6)])
                d = np.array([-1.0, rng.uniform(-0.05, 0.05), rng.uniform(-0.1, 0.1)])
                d /= np.linalg.norm(d)
                rf, _ = O.trace_ray(O.Cloak(variant, form=O.FERMAT), integ, mode, o, d)
                rh, _ = O.trace_ray(O.Cloak(variant, form=O.HAMILTONIAN), integ, mode, o, d)
                assert rf["status"] == rh["status"]
                if rf["status"] in (1, 2):
                    n += 1
                    assert np.max(np.abs(rf["exit_dir"] - rh["exit_dir"])) < 1e-8
                    assert np.max(np.abs(rf["exit_pos"] - rh["exit_pos"])) < 1e-8
                    assert abs(rf["weight"] - rh["weight"]) < 1e-8
    assert n > 15


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
def test_hamiltonian_trace_cloaks_in_plane_rays(variant):
    integ = O.Integrator(O.DP45, 1e-11, 2_000_000)
    for b in (0.2, 0.55, 0.9):
        o = np.array([-4.0, b, 0.0])
        d = np.array([1.0, 0.0, 0.0])
        rec, _ = O.trace_ray(O.Cloak(variant, form=O.HAMILTONIAN), integ, O.EXTRAORDINARY, o, d)
        assert rec["status"] == 1
        assert np.max(np.abs(rec["exit_dir"] - d)) < 1e-9
        assert abs(rec["exit_pos"][1] - b) < 1e-9 and abs(rec["exit_pos"][0] - math.sqrt(1 - b * b)) < 1e-9
        assert abs(rec["tof"] - 2 * math.sqrt(1 - b * b)) < 1e-9
