"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself:
published values (tests/golden), closed forms derived from Eqs. 2, 6-8, 13-15,
textbook Fresnel formulas (isotropic limit of Sect. 3), conservation laws of the
axisymmetric medium, energy conservation (Sect. 3: R = 1 - T), reciprocity,
time reversal and the convergence order of RK4 (Sect. 4).
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
R1, R2, H = 0.5, 1.0, 2.0
K = (R2 / (R2 - R1)) ** 2


def angle(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return math.atan2(np.linalg.norm(np.cross(a, b)), float(np.dot(a, b)))


def lateral_entry(o, d):
    """first intersection of o + s d with r = R2 (test-side geometry)."""
    a = d[0] ** 2 + d[1] ** 2
    b = o[0] * d[0] + o[1] * d[1]
    c = o[0] ** 2 + o[1] ** 2 - R2 ** 2
    s = (-b - math.sqrt(b * b - a * c)) / a
    return o + s * d


def make_ray(L, kz, theta0=0.3, z0=0.0):
    """vacuum ray that enters the side face at azimuth theta0, height z0 with
    tangential wave-vector components d_theta = L / R2 and d_z = kz."""
    dt = L / R2
    dr = -math.sqrt(1.0 - dt * dt - kz * kz)
    rh = np.array([math.cos(theta0), math.sin(theta0), 0.0])
    th = np.array([-math.sin(theta0), math.cos(theta0), 0.0])
    d = dr * rh + dt * th + kz * np.array([0.0, 0.0, 1.0])
    p = R2 * rh + np.array([0, 0, z0])
    return p - 0.5 * d, d, p


def exit_from_angles(theta_in, z_in, dtheta, dz, L, kz):
    th = theta_in + dtheta
    rh = np.array([math.cos(th), math.sin(th), 0.0])
    tv = np.array([-math.sin(th), math.cos(th), 0.0])
    pos = R2 * rh + np.array([0, 0, z_in + dz])
    dt = L / R2
    d = math.sqrt(1 - dt * dt - kz * kz) * rh + dt * tv + np.array([0, 0, kz])
    return pos, d


# ---------------------------------------------------------------- published values
def test_splitmix64_published_sequence():
    vals = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt")) if l.startswith("0x")]
    g = 0x9E3779B97F4A7C15
    for n, v in enumerate(vals):
        assert O.splitmix64((n * g) & (2 ** 64 - 1)) == v


def test_uniform_statistics():
    u = np.array([O.uniform(7, p, s, d) for p in range(4000) for s in range(4) for d in range(2)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1.0 / 12.0) < 0.005


def test_paper_geometry_golden():
    g = dict(l.split() for l in open(os.path.join(GOLD, "paper_geometry.txt")) if l[0] != "#")
    a, b = float(g["a"]), float(g["b"])
    c = O.Cloak(O.RADIAL, R1=a, R2=b, H=0.2)
    for r in (0.06, 0.08, 0.1):
        eps, eo, ee, ch = O.permittivity(c, [r, 0.0, 0.0])
        assert eo == pytest.approx(float(g["K"]), rel=1e-15)
        assert math.sqrt(eo) == pytest.approx(float(g["n_o_radial"]), rel=1e-15)
    # radial ordinary rays: right side of Eq. 2 vanishes (Sect. 4)
    y = [0.07, 0.02, 0.01, 0.2, -0.3, 0.1]
    assert np.abs(O.rhs(c, O.ORDINARY, y)[3:]).max() == 0.0


# ---------------------------------------------------------------- material (Eqs. 7, 13-15)
@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
def test_reduced_parameters_match_ideal_cloak(variant):
    """Sect. 4: eps'_r mu'_z = eps_r mu_z and eps'_theta mu'_z = eps_theta mu_z with the
    ideal parameters of Eq. 13 and mu' = 1."""
    c = O.Cloak(variant)
    for r in np.linspace(0.55, 1.0, 7):
        th = 0.7
        x = [r * math.cos(th), r * math.sin(th), 0.3]
        eps, eo, ee, ch = O.permittivity(c, x)
        rh = np.array([math.cos(th), math.sin(th), 0])
        tv = np.array([-math.sin(th), math.cos(th), 0])
        e_r = rh @ eps @ rh
        e_t = tv @ eps @ tv
        ideal_er, ideal_et = (r - R1) / r, r / (r - R1)
        ideal_mz = (R2 / (R2 - R1)) ** 2 * (r - R1) / r
        assert e_r == pytest.approx(ideal_er * ideal_mz, rel=1e-13)
        assert e_t == pytest.approx(ideal_et * ideal_mz, rel=1e-13)
        # the free component is the other choice: Eq. 14 sets it to eps'_theta, Eq. 15 to eps'_r
        e_z = eps[2, 2]
        assert e_z == pytest.approx(e_t if variant == O.RADIAL else e_r, rel=1e-13)
    # at the outer radius the graded component equals one
    eps, eo, ee, ch = O.permittivity(c, [R2, 0, 0])
    assert eps[0, 0] == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
def test_aux_matrix_structure(variant):
    """Eq. 7: M eps = n_o^2 n_e^2 I; M c = eps_o c, M t = eps_e t for t perpendicular to c."""
    c = O.Cloak(variant)
    rng = np.random.default_rng(1)
    for _ in range(10):
        r = rng.uniform(0.55, 1.0)
        th = rng.uniform(0, 2 * math.pi)
        x = [r * math.cos(th), r * math.sin(th), rng.uniform(-1, 1)]
        M, dM = O.aux_matrix(c, x)
        eps, eo, ee, ch = O.permittivity(c, x)
        np.testing.assert_allclose(M @ eps, eo * ee * np.eye(3), atol=1e-12 * eo * ee)
        np.testing.assert_allclose(M @ ch, eo * ch, atol=1e-12)
        t = np.cross(ch, [0.1, 0.2, 0.9])
        t /= np.linalg.norm(t)
        np.testing.assert_allclose(M @ t, ee * t, atol=1e-12)
        np.testing.assert_allclose(M @ O.aux_inverse(c, x), np.eye(3), atol=1e-13)


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
def test_grad_M_finite_difference(variant):
    c = O.Cloak(variant)
    rng = np.random.default_rng(2)
    for _ in range(10):
        r = rng.uniform(0.52, 1.2)
        th = rng.uniform(0, 2 * math.pi)
        x = np.array([r * math.cos(th), r * math.sin(th), rng.uniform(-1, 1)])
        M, dM = O.aux_matrix(c, x)
        hstep = 1e-6
        for k in range(3):
            e = np.zeros(3)
            e[k] = hstep
            fd = (O.aux_matrix(c, x + e)[0] - O.aux_matrix(c, x - e)[0]) / (2 * hstep)
            scale = max(1.0, np.abs(dM[k]).max())
            assert np.abs(fd - dM[k]).max() < 1e-7 * scale


# ---------------------------------------------------------------- equations of motion (Eqs. 2, 8)
def test_eq8_reduces_to_eq2_for_isotropic_M():
    """Sect. 2: for M = n^2 I (ordinary ray), Eq. 8 coincides with Eq. 2."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        n = rng.uniform(0.5, 3.0)
        gn = rng.normal(size=3)
        v = rng.normal(size=3)
        M = n * n * np.eye(3)
        dM = np.stack([2 * n * gn[k] * np.eye(3) for k in range(3)])
        np.testing.assert_allclose(O.eq8_accel(np.linalg.inv(M), dM, v), O.eq2_accel(n, gn, v), rtol=1e-12,
                                   atol=1e-12)


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
@pytest.mark.parametrize("mode", [O.ORDINARY, O.EXTRAORDINARY])
def test_eom_is_hamiltonian_flow(variant, mode):
    """Eq. 6 with H(x, k) = (k^T M^{-1} k - 1)/2: the ray equation must give
    d(Mv)/dt = -dH/dx at fixed k.  Both sides by finite differences of M only."""
    c = O.Cloak(variant)
    rng = np.random.default_rng(4)

    def Mof(x):
        if mode == O.EXTRAORDINARY:
            return O.aux_matrix(c, x)[0]
        return O.permittivity(c, x)[1] * np.eye(3)

    for _ in range(10):
        r = rng.uniform(0.6, 1.0)
        th = rng.uniform(0, 2 * math.pi)
        x = np.array([r * math.cos(th), r * math.sin(th), rng.uniform(-1, 1)])
        v = rng.normal(size=3) * 0.5
        a = O.rhs(c, mode, np.concatenate([x, v]))[3:]
        M = Mof(x)
        k = M @ v
        hs = 1e-6
        dHdx = np.zeros(3)
        for i in range(3):
            e = np.zeros(3)
            e[i] = hs
            Hp = 0.5 * k @ np.linalg.solve(Mof(x + e), k)
            Hm = 0.5 * k @ np.linalg.solve(Mof(x - e), k)
            dHdx[i] = (Hp - Hm) / (2 * hs)
        dMdt = (Mof(x + hs * v) - Mof(x - hs * v)) / (2 * hs)
        dkdt = dMdt @ v + M @ a
        np.testing.assert_allclose(dkdt, -dHdx, rtol=2e-6, atol=2e-7 * max(1, np.abs(dkdt).max()))


# ---------------------------------------------------------------- interface (Sect. 3, Eqs. 9-12)
def fresnel(i, n):
    ci = math.cos(i)
    st = math.sin(i) / n
    ct = math.sqrt(1 - st * st)
    rs = (ci - n * ct) / (ci + n * ct)
    rp = (n * ci - ct) / (n * ci + ct)
    return 1 - rs * rs, 1 - rp * rp, math.asin(st)


@pytest.mark.parametrize("inc_deg", [0.0, 15.0, 40.0, 65.0, 85.0])
def test_isotropic_limit_snell_fresnel(inc_deg):
    n = 1.5
    c = O.Cloak(O.TEST_CONST, R1=0.0, eps_o=n * n, eps_e=n * n, c_hat=(0.3, 0.4, 0.866))
    i = math.radians(inc_deg)
    nh = np.array([0.0, 0.0, 1.0])
    d = np.array([math.sin(i), 0.0, -math.cos(i)])
    Ts, Tp, t = fresnel(i, n)
    T = O.transmission_in(c, [0.2, 0.1, 1.0], nh, d)
    assert T["To_s"] + T["Te_s"] == pytest.approx(Ts, abs=1e-12)
    assert T["To_p"] + T["Te_p"] == pytest.approx(Tp, abs=1e-12)
    for mode in (O.ORDINARY, O.EXTRAORDINARY):
        k, v = O.refract_into(c, mode, [0.2, 0.1, 1.0], nh, d - (d @ nh) * nh)
        assert np.linalg.norm(k) == pytest.approx(n, rel=1e-12)
        assert angle(k, -nh) == pytest.approx(t, abs=1e-12)  # Snell
        np.testing.assert_allclose(v, k / (n * n), atol=1e-14)


def test_normal_incidence_closed_form():
    """Normal incidence on the side face at r = R2 (textbook single-interface
    T = 4n/(1+n)^2).  Radial: k parallel to c, both modes see n = 2.  Azimuthal:
    the ordinary wave sees n_o = 1, the extraordinary n_e = 2."""
    x = np.array([R2, 0, 0])
    nh = np.array([1.0, 0, 0])
    d = -nh
    t2 = 4 * 2 / 9.0
    T = O.transmission_in(O.Cloak(O.RADIAL), x, nh, d)
    assert T["To"] + T["Te"] == pytest.approx(t2, abs=1e-12)
    T = O.transmission_in(O.Cloak(O.AZIMUTHAL), x, nh, d)
    assert T["To"] == pytest.approx(0.5, abs=1e-12)
    assert T["Te"] == pytest.approx(0.5 * t2, abs=1e-12)


FACES = [
    ("radial side", O.RADIAL, [R2, 0, 0.2], [1, 0, 0]),
    ("azimuthal side", O.AZIMUTHAL, [R2 * 0.6, R2 * 0.8, -0.3], [0.6, 0.8, 0]),
    ("radial cap", O.RADIAL, [0.45, 0.5, 1.0], [0, 0, 1]),
    ("azimuthal cap", O.AZIMUTHAL, [0.55, -0.4, -1.0], [0, 0, -1]),
]


def random_inward(rng, nh):
    while True:
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if d @ nh < -0.02:
            return d


@pytest.mark.parametrize("name,variant,x,n", FACES)
def test_energy_conservation_entry(name, variant, x, n):
    """Sect. 3: reflection = 1 - transmission, for each incident polarisation."""
    c = O.Cloak(variant)
    rng = np.random.default_rng(5)
    nh = np.array(n, float)
    for _ in range(25):
        d = random_inward(rng, nh)
        T = O.transmission_in(c, x, nh, d)
        assert T["R_s"] + T["To_s"] + T["Te_s"] == pytest.approx(1.0, abs=1e-11)
        assert T["R_p"] + T["To_p"] + T["Te_p"] == pytest.approx(1.0, abs=1e-11)


def test_energy_conservation_tilted_axis():
    c = O.Cloak(O.TEST_CONST, R1=0.0, eps_o=2.2, eps_e=3.1, c_hat=(0.5, -0.3, 0.81))
    rng = np.random.default_rng(6)
    nh = np.array([0.0, 0.0, 1.0])
    for _ in range(25):
        d = random_inward(rng, nh)
        T = O.transmission_in(c, [0.1, 0.2, 1.0], nh, d)
        assert T["R_s"] + T["To_s"] + T["Te_s"] == pytest.approx(1.0, abs=1e-11)
        assert T["R_p"] + T["To_p"] + T["Te_p"] == pytest.approx(1.0, abs=1e-11)
        for mode in (O.ORDINARY, O.EXTRAORDINARY):
            k, v = O.refract_into(c, mode, [0.1, 0.2, 1.0], nh, d - (d @ nh) * nh)
            # wave vector on the index surface, inward ray velocity
            M = O.aux_matrix(c, [0.1, 0.2, 1.0])[0] if mode else 2.2 * np.eye(3)
            assert k @ np.linalg.solve(M, k) == pytest.approx(1.0, abs=1e-12)
            assert v @ nh < 0


def outward_wave(c, mode, x, nh, kt):
    k, v = O.refract_into(c, mode, x, nh, -kt)
    return -k


@pytest.mark.parametrize("name,variant,x,n", FACES)
def test_energy_conservation_exit_and_reciprocity(name, variant, x, n):
    """Exit face (Sect. 3, last paragraph): T + R_o + R_e = 1.  Reciprocity: the
    power carried from vacuum (summed over s and p) into a mode equals the power
    that the time-reversed mode sends back into vacuum."""
    c = O.Cloak(variant)
    rng = np.random.default_rng(7)
    nh = np.array(n, float)
    checked = 0
    for _ in range(40):
        d = random_inward(rng, nh)
        kt = d - (d @ nh) * nh
        T = O.transmission_in(c, x, nh, d)
        for mode in (O.ORDINARY, O.EXTRAORDINARY):
            w = O.refract_into(c, mode, x, nh, kt)
            if w is None:
                continue
            k, v = w
            ok, Tout, Ro, Re = O.transmission_out(c, mode, x, nh, -k)
            assert ok
            assert Tout + Ro + Re == pytest.approx(1.0, abs=1e-11)
            tin = T["To_s"] + T["To_p"] if mode == O.ORDINARY else T["Te_s"] + T["Te_p"]
            assert Tout == pytest.approx(tin, abs=1e-11)
            checked += 1
    assert checked > 15


def test_section5_main_section_claim():
    """Sect. 5: with k in the plane containing the cylinder axis and the face
    normal, the radial cloak puts D_e in that plane, the azimuthal cloak puts
    D_e perpendicular to it; with k in the design plane D_e stays in the design
    plane for both.  Also D = eps E = -k x (k x E) (Maxwell) for both modes."""
    x = np.array([R2, 0, 0.1])
    nh = np.array([1.0, 0, 0])
    for alpha in (0.2, 0.6, 1.0):
        d_h = np.array([-math.cos(alpha), 0.0, math.sin(alpha)])   # plane containing the axis (xz)
        d_v = np.array([-math.cos(alpha), math.sin(alpha), 0.0])   # design plane (xy)
        for variant in (O.RADIAL, O.AZIMUTHAL):
            c = O.Cloak(variant)
            k, v = O.refract_into(c, O.EXTRAORDINARY, x, nh, d_h - (d_h @ nh) * nh)
            D, E, Hh = O.mode_fields(c, O.EXTRAORDINARY, x, k)
            D /= np.linalg.norm(D)
            if variant == O.RADIAL:
                assert abs(D[1]) < 1e-12
            else:
                assert abs(D[0]) < 1e-12 and abs(D[2]) < 1e-12
            k, v = O.refract_into(c, O.EXTRAORDINARY, x, nh, d_v - (d_v @ nh) * nh)
            D, E, Hh = O.mode_fields(c, O.EXTRAORDINARY, x, k)
            assert abs(D[2]) < 1e-12 * np.linalg.norm(D)
            for mode in (O.ORDINARY, O.EXTRAORDINARY):
                k, v = O.refract_into(c, mode, x, nh, d_h - (d_h @ nh) * nh)
                D, E, Hh = O.mode_fields(c, mode, x, k)
                np.testing.assert_allclose(D, -np.cross(k, np.cross(k, E)), atol=1e-12 * np.linalg.norm(D))
                assert abs(D @ k) < 1e-12 * np.linalg.norm(D) * np.linalg.norm(k)


# ---------------------------------------------------------------- whole rays (Sect. 4)
def trace(c, mode, o, d, kind=O.RK4, h=1e-3, path=0):
    return O.trace_ray(c, O.Integrator(kind, h), mode, o, d, path_cap=path)


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
@pytest.mark.parametrize("p", [0.2, 0.5, 0.85])
def test_inplane_perfect_cloaking(variant, p):
    """Sect. 4: in-plane rays of in-plane polarisation (extraordinary) are cloaked
    perfectly: the exit ray continues the entry line, leaves at the far
    intersection of that line with r = R2, after the vacuum time of flight."""
    c = O.Cloak(variant)
    o = np.array([3.0, p, 0.0])
    d = np.array([-1.0, 0.0, 0.0])
    rec, _ = trace(c, O.EXTRAORDINARY, o, d)
    assert O.STATUS[rec["status"]] == "EXITED"
    far = np.array([-math.sqrt(R2 * R2 - p * p), p, 0.0])
    assert angle(rec["exit_dir"], d) < 1e-9
    assert np.abs(rec["exit_pos"] - far).max() < 1e-9
    assert rec["tof"] == pytest.approx(2 * math.sqrt(R2 * R2 - p * p), abs=1e-9)


@pytest.mark.parametrize("L,kz", [(0.3, 0.2), (-0.6, -0.35), (0.85, 0.5), (0.1, 0.0)])
def test_azimuthal_extraordinary_closed_form(L, kz):
    """Azimuthal e-ray (Eq. 8 with M = diag(K, f, K)): with u = r - R1 the motion is
    a straight line in (sqrt(K - k_z^2) u, theta) traversed at speed (K-k_z^2)/K."""
    c = O.Cloak(O.AZIMUTHAL)
    o, d, p = make_ray(L, kz, theta0=0.3, z0=-0.2 * np.sign(kz))
    U = R2 - R1
    Kp = K - kz * kz
    root = math.sqrt(Kp * U * U - L * L)
    dth = math.copysign(2 * math.acos(abs(L) / (U * math.sqrt(Kp))), L)
    dz = 2 * kz * root / Kp
    tof = 2 * K * root / Kp
    pos, dexp = exit_from_angles(0.3, p[2], dth, dz, L, kz)
    rec, _ = trace(c, O.EXTRAORDINARY, o, d, O.DP45, 1e-12)
    assert O.STATUS[rec["status"]] == "EXITED"
    assert angle(rec["exit_dir"], dexp) < 5e-10
    assert np.abs(rec["exit_pos"] - pos).max() < 5e-10
    assert rec["tof"] == pytest.approx(tof, abs=5e-10)


def quad_exit(L, kz, which):
    """Exit state of a radial e-ray or azimuthal o-ray by quadrature.
    R(u) = K u^2 - L^2 - k_z^2 (u + R1)^2; substitution u = u_t + w^2."""
    from scipy.integrate import quad
    A = K - kz * kz
    B = -2 * kz * kz * R1
    C = -(L * L + kz * kz * R1 * R1)
    disc = math.sqrt(B * B - 4 * A * C)
    ut, u2 = (-B + disc) / (2 * A), (-B - disc) / (2 * A)
    U = R2 - R1
    W = math.sqrt(U - ut)

    def I(g):
        f = lambda w: g(ut + w * w) * 2.0 / math.sqrt(A * (w * w + ut - u2))
        return quad(f, 0.0, W, epsabs=1e-14, epsrel=1e-13, limit=200)[0]

    if which == "radial_e":
        tof = 2 * I(lambda u: K * u)
        dth = 2 * L * I(lambda u: 1.0 / u)
        dz = 2 * kz * I(lambda u: (u + R1) ** 2 / u)
    else:
        tof = 2 * I(lambda u: K * u * u / (u + R1))
        dth = 2 * L * I(lambda u: 1.0 / (u + R1))
        dz = 2 * kz * I(lambda u: u + R1)
    return tof, dth, dz


@pytest.mark.parametrize("which,variant,mode", [("radial_e", O.RADIAL, O.EXTRAORDINARY),
                                                 ("azim_o", O.AZIMUTHAL, O.ORDINARY)])
@pytest.mark.parametrize("L,kz", [(0.3, 0.25), (-0.7, 0.4), (0.5, -0.3)])
def test_quadrature_closed_form(which, variant, mode, L, kz):
    """Radial e-ray (M = diag(K, f, f)) and azimuthal o-ray (M = f I): conserved
    k_z and L_z reduce the motion to 1-D integrals over u = r - R1."""
    c = O.Cloak(variant)
    o, d, p = make_ray(L, kz, theta0=1.1, z0=-0.15 * np.sign(kz))
    tof, dth, dz = quad_exit(L, kz, which)
    pos, dexp = exit_from_angles(1.1, p[2], dth, dz, L, kz)
    rec, _ = trace(c, mode, o, d, O.DP45, 1e-12)
    assert O.STATUS[rec["status"]] == "EXITED"
    assert angle(rec["exit_dir"], dexp) < 2e-9
    assert np.abs(rec["exit_pos"] - pos).max() < 2e-9
    assert rec["tof"] == pytest.approx(tof, abs=2e-9)


@pytest.mark.parametrize("L,kz", [(0.2, 0.1), (-0.45, -0.2), (0.8, 0.3)])
def test_radial_ordinary_is_lens_with_mirror(L, kz):
    """Sect. 4: radial o-rays see n_o = 2 everywhere, go straight, all reach the
    metal cylinder (single mirror ray) and leave like a cylindrical lens."""
    c = O.Cloak(O.RADIAL)
    o, d, p = make_ray(L, kz, theta0=-0.4, z0=0.1)
    n = 2.0
    nh = np.array([p[0], p[1], 0]) / R2
    kt = d - (d @ nh) * nh
    k = kt - math.sqrt(n * n - kt @ kt) * nh
    u = k / n
    a = u[0] ** 2 + u[1] ** 2
    b = p[0] * u[0] + p[1] * u[1]
    cc = p[0] ** 2 + p[1] ** 2 - R1 * R1
    s1 = (-b - math.sqrt(b * b - a * cc)) / a
    q = p + s1 * u
    nm = np.array([q[0], q[1], 0]) / R1
    u2 = u - 2 * (u @ nm) * nm
    b2 = q[0] * u2[0] + q[1] * u2[1]
    c2 = R1 * R1 - R2 * R2
    s2 = (-b2 + math.sqrt(b2 * b2 - a * c2)) / a
    e = q + s2 * u2
    ne = np.array([e[0], e[1], 0]) / R2
    ke = n * u2
    kte = ke - (ke @ ne) * ne
    dexp = kte + math.sqrt(1 - kte @ kte) * ne
    rec, _ = trace(c, O.ORDINARY, o, d)
    assert O.STATUS[rec["status"]] == "HIT_METAL_EXITED"
    assert angle(rec["exit_dir"], dexp) < 1e-11
    assert np.abs(rec["exit_pos"] - e).max() < 1e-11
    assert rec["tof"] == pytest.approx((s1 + s2) * n, abs=1e-11)  # ray speed 1/n


def test_rk4_fourth_order_convergence():
    c = O.Cloak(O.AZIMUTHAL)
    L, kz = 0.35, 0.2
    o, d, p = make_ray(L, kz, theta0=0.0, z0=-0.1)
    U, Kp = R2 - R1, K - kz * kz
    root = math.sqrt(Kp * U * U - L * L)
    dth = 2 * math.acos(L / (U * math.sqrt(Kp)))
    pos, dexp = exit_from_angles(0.0, p[2], dth, 2 * kz * root / Kp, L, kz)
    errs = []
    for h in (8e-3, 4e-3, 2e-3):
        rec, _ = trace(c, O.EXTRAORDINARY, o, d, O.RK4, h)
        errs.append(np.abs(rec["exit_pos"] - pos).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 10 < r1 < 24 and 10 < r2 < 24, errs


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
@pytest.mark.parametrize("mode", [O.ORDINARY, O.EXTRAORDINARY])
def test_conservation_along_path(variant, mode):
    """Axisymmetric, z-invariant medium: k_z and L_z = (x x k)_z are conserved, and
    the ray Hamiltonian v^T M v = 1 (Eq. 6 with the dispersion relation)."""
    c = O.Cloak(variant)
    o, d, p = make_ray(0.4, 0.3, theta0=0.5, z0=-0.3)
    rec, path = trace(c, mode, o, d, O.RK4, 1e-3, path=100000)
    assert len(path) > 100
    kz0 = d[2]
    L0 = o[0] * d[1] - o[1] * d[0]
    for row in path[:: max(1, len(path) // 200)]:
        x, v = row[1:4], row[4:7]
        M = O.aux_matrix(c, x)[0] if mode == O.EXTRAORDINARY else O.permittivity(c, x)[1] * np.eye(3)
        k = M @ v
        assert v @ M @ v == pytest.approx(1.0, abs=1e-10)
        assert k[2] == pytest.approx(kz0, abs=1e-10)
        assert x[0] * k[1] - x[1] * k[0] == pytest.approx(L0, abs=1e-10)


@pytest.mark.parametrize("variant", [O.RADIAL, O.AZIMUTHAL])
@pytest.mark.parametrize("mode", [O.ORDINARY, O.EXTRAORDINARY])
def test_time_reversal(variant, mode):
    c = O.Cloak(variant)
    o, d, p = make_ray(0.55, -0.25, theta0=2.0, z0=0.2)
    rec, _ = trace(c, mode, o, d, O.DP45, 1e-12)
    e, de = rec["exit_pos"], rec["exit_dir"]
    rec2, _ = trace(c, mode, e + 0.5 * de, -de, O.DP45, 1e-12)
    assert angle(rec2["exit_dir"], -d) < 1e-9
    assert np.abs(rec2["exit_pos"] - p).max() < 1e-9
    assert rec2["tof"] == pytest.approx(rec["tof"], abs=1e-9)
    assert rec2["weight"] == pytest.approx(rec["weight"], abs=1e-12)


def test_paper_statements_about_metal():
    """Sect. 4: all radial o-rays reach the metal cylinder and no radial e-ray does;
    in the azimuthal cloak no ray reaches it."""
    rng = np.random.default_rng(8)
    for _ in range(12):
        L = rng.uniform(-0.9, 0.9)
        kz = rng.uniform(-0.2, 0.2)
        o, d, p = make_ray(L, kz, theta0=rng.uniform(0, 6.28), z0=0.0)
        assert trace(O.Cloak(O.RADIAL), O.ORDINARY, o, d)[0]["status"] == 2
        assert trace(O.Cloak(O.RADIAL), O.EXTRAORDINARY, o, d)[0]["status"] == 1
        assert trace(O.Cloak(O.AZIMUTHAL), O.ORDINARY, o, d)[0]["status"] == 1
        assert trace(O.Cloak(O.AZIMUTHAL), O.EXTRAORDINARY, o, d)[0]["status"] == 1


# ---------------------------------------------------------------- camera and room
def test_camera_geometry():
    cam = O.Camera(eye=(5, 0, 0), hfov_deg=60.0, width=128, height=96)
    w = np.array([-1.0, 0, 0])
    o, dl = O.camera_ray(cam, 0, 47, 0, 1, 0)
    o, dr = O.camera_ray(cam, 127, 47, 0, 1, 0)
    np.testing.assert_allclose(o, [5, 0, 0])
    half = math.atan((1 - 1 / 128) * math.tan(math.radians(30)))
    assert angle(dl, w) == pytest.approx(angle(dr, w), abs=1e-14)
    assert angle(dl, dr) == pytest.approx(2 * math.atan(math.tan(half) * math.cos(angle(dl, w)) / math.cos(half)),
                                          abs=2e-3)
    assert dl[1] < 0 < dr[1]                     # image right = +y when looking along -x with up = +z
    o, dt = O.camera_ray(cam, 64, 0, 0, 1, 0)
    assert dt[2] > 0                             # row 0 at the top


def test_room_tiles():
    c = O.Cloak(O.RADIAL)
    t, rgb = O.shade(c, [0, 0, 0], [0, 0, -1])
    assert t == (4 << 20) | (80 << 10) | 80
    t2, rgb2 = O.shade(c, [1.0 / 16 + 0.125, 0.0 + 1.0 / 16, 0], [0, 0, -1])
    assert t2 == (4 << 20) | (81 << 10) | 80
    assert rgb.min() >= 0.85 * 0.6 - 1e-12 and rgb.max() <= 0.85 + 1e-12     # even tile: light
    assert rgb2.max() <= 0.25 + 1e-12                                        # odd tile: dark
    t3, _ = O.shade(c, [0, 0, 0], [1, 0, 0])
    assert t3 == (0 << 20) | (80 << 10) | 8
    t4, rgb4 = O.shade(c, [0, 0, 0], [0, 0, 1])
    assert t4 == 5 << 20


@pytest.mark.parametrize("p", [0.15, 0.45, 0.8])
def test_inplane_weights_closed_form(p):
    """Eq. 12 for in-plane rays.  Extraordinary (TM, E in the plane): the face sees
    eps_t = 4 along the surface and eps_n = 1 along the normal in both cloaks, so
    k_n = 2 cos(i) and r = (4 cos i - 2 cos i)/(4 cos i + 2 cos i) = 1/3 at every angle:
    weight = 1/2 (8/9)^2 (half of the unpolarised light, two faces).  Ordinary (TE,
    E along z): azimuthal eps_z = 1 at r = R2 (no reflection, weight 1/2); radial
    n_o = 2 (Fresnel T_s at the same internal angle on both faces)."""
    o = np.array([3.0, p, 0.0])
    d = np.array([-1.0, 0.0, 0.0])
    for variant in (O.RADIAL, O.AZIMUTHAL):
        rec, _ = trace(O.Cloak(variant), O.EXTRAORDINARY, o, d)
        assert rec["weight"] == pytest.approx(0.5 * (8.0 / 9.0) ** 2, abs=1e-12)
    rec, _ = trace(O.Cloak(O.AZIMUTHAL), O.ORDINARY, o, d)
    assert rec["weight"] == pytest.approx(0.5, abs=1e-12)
    i = math.asin(p / R2)
    Ts, Tp, t = fresnel(i, 2.0)
    rec, _ = trace(O.Cloak(O.RADIAL), O.ORDINARY, o, d)
    assert rec["weight"] == pytest.approx(0.5 * Ts * Ts, abs=1e-12)


@pytest.mark.parametrize("which,variant,mode,L,kz,tol", [
    ("radial_e", O.RADIAL, O.EXTRAORDINARY, 1e-3, 0.003, 2e-9),
    ("radial_e", O.RADIAL, O.EXTRAORDINARY, -2e-3, -0.004, 2e-9),
    ("azim_o", O.AZIMUTHAL, O.ORDINARY, 2e-4, 0.02, 2e-9),
    ("azim_o", O.AZIMUTHAL, O.ORDINARY, -3e-3, 0.1, 2e-9),
])
def test_near_axis_closed_form(which, variant, mode, L, kz, tol):
    """Rays passing within ~1e-3 of the inner radius, where f = K((r-R1)/r)^2 -> 0
    and one principal value of eps and M vanishes: the oracle must stay accurate
    there.  The entry height is chosen so that the path is centred in z."""
    tof, dth, dz = quad_exit(L, kz, which)
    assert abs(dz) < 1.9
    z0 = -0.5 * dz
    o, d, p = make_ray(L, kz, theta0=1.1, z0=z0)
    pos, dexp = exit_from_angles(1.1, z0, dth, dz, L, kz)
    rec, _ = trace(O.Cloak(variant), mode, o, d, O.DP45, 1e-12)
    assert O.STATUS[rec["status"]] == "EXITED"
    assert angle(rec["exit_dir"], dexp) < tol
    assert np.abs(rec["exit_pos"] - pos).max() < tol
    assert rec["tof"] == pytest.approx(tof, abs=tol)


@pytest.mark.parametrize("L,kz,tol", [(-3e-3, 0.1, 1e-10), (2e-4, 0.02, 1e-8)])
def test_near_axis_azimuthal_extraordinary(L, kz, tol):
    """Azimuthal e-ray with impact parameter down to 2e-4: the ray speed near the
    turning point grows like 1/L (superluminal region, Sect. 6)."""
    c = O.Cloak(O.AZIMUTHAL)
    U, Kp = R2 - R1, K - kz * kz
    root = math.sqrt(Kp * U * U - L * L)
    dth = math.copysign(2 * math.acos(abs(L) / (U * math.sqrt(Kp))), L)
    dz = 2 * kz * root / Kp
    o, d, p = make_ray(L, kz, theta0=0.3, z0=-0.5 * dz)
    pos, dexp = exit_from_angles(0.3, -0.5 * dz, dth, dz, L, kz)
    rec, _ = trace(c, O.EXTRAORDINARY, o, d, O.DP45, 1e-12)
    assert O.STATUS[rec["status"]] == "EXITED"
    assert angle(rec["exit_dir"], dexp) < tol
    assert rec["tof"] == pytest.approx(2 * K * root / Kp, abs=tol)


def test_all_radial_ordinary_rays_reach_metal_with_dp45():
    """Sect. 4: every radial ordinary ray that enters laterally reaches the metal cylinder --
    also with the adaptive integrator, whose steps grow without bound on these straight rays."""
    rng = np.random.default_rng(9)
    c = O.Cloak(O.RADIAL)
    for _ in range(40):
        L = rng.uniform(-0.97, 0.97)
        kz = rng.uniform(-0.1, 0.1)
        o, d, p = make_ray(L, kz, theta0=rng.uniform(0, 6.28), z0=0.0)
        for tol in (1e-9, 1e-6):
            rec, _ = trace(c, O.ORDINARY, o, d, O.DP45, tol)
            assert O.STATUS[rec["status"]] == "HIT_METAL_EXITED", (L, kz, tol)
