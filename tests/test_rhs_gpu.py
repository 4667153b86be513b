"""The right-hand side of the ray equations as the GPU integrators evaluate it (cylindrical closed form,
FP64 reciprocal and 1/sqrt from the hardware seeds plus one Newton-Raphson step each) against the oracle's
literal evaluation of Eq. 8 / Eq. 2 (Fermat form) and of the Hamiltonian form, state by state."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

R1, R2, H = 0.5, 1.0, 2.0


@pytest.fixture(scope="module")
def ck():
    import torch
    from paper_1209_6038_gb300 import build, cloak
    build.build()
    cloak.load()
    torch.cuda.init()
    return cloak


def states(n, rmin, rmax, seed):
    rng = np.random.default_rng(seed)
    r = rmin + (rmax - rmin) * rng.random(n)
    th = 2 * np.pi * rng.random(n)
    y = np.empty((n, 6))
    y[:, 0], y[:, 1] = r * np.cos(th), r * np.sin(th)
    y[:, 2] = (rng.random(n) - 0.5) * H
    y[:, 3:] = rng.normal(size=(n, 3))
    return y


def compare(ck, variant, mode, form, y):
    import torch
    c = ck.Cloak(variant, R1, R2, H).formulation(form)
    g = c.eval_rhs(mode, torch.from_numpy(y)).cpu().numpy()
    c.close()
    oc = O.Cloak(variant, R1, R2, H)
    f = O.rhs if form == ck.FORM_FERMAT else O.rhs_hamiltonian
    o = np.array([f(oc, mode, row) for row in y])
    scale = np.abs(o).max(axis=1)
    return np.abs(g - o).max(axis=1) / scale


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("variant,mode", [(0, 1), (1, 0), (1, 1), (0, 0)])
def test_rhs_matches_the_oracle_away_from_the_inner_radius(ck, form, variant, mode):
    """u = r - R1 >= 0.2: the closed form and the literal evaluation differ by rounding only (a few 2^-53);
    a reciprocal or 1/sqrt good to 2^-45 only would already fail."""
    if variant == 0 and mode == 0 and form == 0:
        y = states(512, R1 + 0.2, R2, 3)
        import torch
        c = ck.Cloak(variant, R1, R2, H)
        g = c.eval_rhs(mode, torch.from_numpy(y)).cpu().numpy()
        c.close()
        assert np.array_equal(g[:, :3], y[:, 3:]) and np.all(g[:, 3:] == 0.0)  # straight lines (Sect. 4)
        return
    rel = compare(ck, variant, mode, form, states(2048, R1 + 0.2, R2, 7 + variant + 2 * mode + 4 * form))
    assert rel.max() < 2e-14


# ---- near the inner radius the oracle's literal Cartesian evaluation of Eq. 8 loses digits (its terms
# cancel to O(r - R1) before the 1/f ~ 1/(r - R1)^2 factor); there the GPU's result is checked against
# what the physics fixes instead: along the ray k_z, L_z = (x cross k)_z and the Hamiltonian are conserved
# (rotation and translation symmetry of both cloaks; time independence).  For the Fermat form (k = M v,
# H = v^T M v) these give three linear equations in dv/dt that fix it wherever v_r != 0.  The auxiliary
# matrix M(x) of Eq. 7 with Eq. 14 / 15 is evaluated in extended precision, its derivative along v by the
# complex step (exact to rounding).

LD, CLD = np.longdouble, np.clongdouble


def aux_matrix(variant, mode, X):
    x, y = X[:, 0], X[:, 1]
    r = np.sqrt(x * x + y * y)
    one, zero = np.ones_like(r), np.zeros_like(r)
    rh = np.stack([x / r, y / r, zero], 1)
    th = np.stack([-y / r, x / r, zero], 1)
    zh = np.stack([zero, zero, one], 1)
    K = LD((R2 / (R2 - R1)) ** 2)
    f = K * ((r - LD(R1)) / r) ** 2

    def outer(a, b):
        return a[:, :, None] * b[:, None, :]
    if mode == 0:  # azimuthal ordinary: M = eps_o I = f I
        return f[:, None, None] * (outer(rh, rh) + outer(th, th) + outer(zh, zh))
    if variant == 0:  # radial extraordinary: diag(K, f, f)
        return K * outer(rh, rh) + f[:, None, None] * (outer(th, th) + outer(zh, zh))
    return K * outer(rh, rh) + f[:, None, None] * outer(th, th) + K * outer(zh, zh)  # diag(K, f, K)


def directional(variant, mode, X, D):
    """(D . grad) M at X, by the complex step."""
    hs = LD(1e-40)
    return np.imag(aux_matrix(variant, mode, X.astype(CLD) + 1j * hs * D.astype(CLD))) / hs


def mv(A, b):
    return np.einsum("nij,nj->ni", A, b)


def norm(a):
    return np.sqrt(np.sum(a * a, 1))


def cz(a, b):
    return a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]


def conservation_residuals(variant, mode, form, y, dy):
    X, S = y[:, :3].astype(LD), y[:, 3:].astype(LD)
    D, E = dy[:, :3].astype(LD), dy[:, 3:].astype(LD)
    M = aux_matrix(variant, mode, X)
    if form == 0:  # state (x, v): D = v, E = dv/dt; k = M v
        V = S
        dM = directional(variant, mode, X, V)
        Mv, Ma, dMv = mv(M, V), mv(M, E), mv(dM, V)
        res = [np.abs(D - V).max(1) / norm(V),
               np.abs(dMv[:, 2] + Ma[:, 2]) / (norm(dMv) + norm(Ma)),                                 # k_z
               np.abs(cz(V, Mv) + cz(X, dMv) + cz(X, Ma)) / (norm(V) * norm(Mv) + norm(X) * (norm(dMv) + norm(Ma))),
               np.abs(2 * np.sum(V * Ma, 1) + np.sum(V * dMv, 1)) / (norm(V) * (2 * norm(Ma) + norm(dMv)))]
    else:  # state (x, k): D = dx/dt = M^-1 k, E = dk/dt; dH/dt = -D^T (D . grad M) D + 2 D . E
        Kv = S
        dM = directional(variant, mode, X, D)
        MD, dMD = mv(M, D), mv(dM, D)
        res = [np.abs(MD - Kv).max(1) / norm(Kv),
               np.abs(E[:, 2]) / (norm(E) + 0.5 * norm(dMD) * norm(D)),                                 # k_z
               np.abs(cz(D, Kv) + cz(X, E)) / (norm(D) * norm(Kv) + norm(X) * norm(E)),
               np.abs(-np.sum(D * dMD, 1) + 2 * np.sum(D * E, 1)) / (norm(D) * (norm(dMD) + 2 * norm(E)))]
    return np.max(np.stack([r.astype(float) for r in res], 1), 1)


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("variant,mode", [(0, 1), (1, 0), (1, 1)])
def test_rhs_conserves_kz_lz_and_h_down_to_the_inner_radius(ck, form, variant, mode):
    """u = r - R1 from 1e-6 to 0.5.  The bar is what rounding allows: u = r - R1 itself carries ~1e-16 / u
    relative error; in the Hamiltonian form dx/dt = M^-1 k is ~1/u^2 along theta, so its Cartesian rounding
    alone moves the radial component by ~1e-16 / u^2 (an exactly rounded result shows the same).
    A 1e-3 relative error in one component gives residuals of 1e-4 or more."""
    import torch
    rng = np.random.default_rng(11 + variant + 2 * mode + 4 * form)
    n = 1024
    u = 10.0 ** rng.uniform(-6, np.log10(R2 - R1), n)
    th = 2 * np.pi * rng.random(n)
    y = np.stack([(R1 + u) * np.cos(th), (R1 + u) * np.sin(th), (rng.random(n) - 0.5) * H,
                  *rng.normal(size=(3, n))], 1)
    c = ck.Cloak(variant, R1, R2, H).formulation(form)
    dy = c.eval_rhs(mode, torch.from_numpy(y)).cpu().numpy()
    c.close()
    res = conservation_residuals(variant, mode, form, y, dy)
    assert np.all(res < 1e-14 + 2e-15 / u + (1e-15 / u ** 2 if form == 1 else 0.0))
    # the check itself: the oracle's own derivative passes it where its evaluation is well conditioned,
    # and a perturbed one fails
    oc = O.Cloak(variant, R1, R2, H)
    far = u > 0.1
    f = O.rhs if form == 0 else O.rhs_hamiltonian
    do = np.array([f(oc, mode, row) for row in y[far]])
    assert np.all(conservation_residuals(variant, mode, form, y[far], do) < 1e-12)
    bad = do.copy()
    bad[:, 3] *= 1.001
    assert np.median(conservation_residuals(variant, mode, form, y[far], bad)) > 1e-5


def test_rhs_arguments(ck):
    import torch
    c = ck.Cloak(ck.RADIAL)
    y = torch.zeros((4, 6), dtype=torch.float64, device="cuda")
    with pytest.raises(ck.CloakError):
        c.eval_rhs(7, y)
    c.close()
    t = ck.Cloak(ck.TEST_UNIAXIAL_CONST, R1=0.0)
    with pytest.raises(ck.CloakError):
        t.eval_rhs(ck.POL_ORDINARY, y)
    t.close()
