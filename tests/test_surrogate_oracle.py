"""Pins of the surrogate part of the oracle (oracle/surrogate_oracle.c) against things other than itself:
PyTorch's own GELU, linear layers, autograd and Adam (independent library implementations), central
differences, distribution moments of the seeded training set, and rays traced by the oracle's
integrator (conservation of k_z and L_z, in-plane perfect cloaking)."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")

SMALL = (7, 16, 12, 5)


def rand_params(dims, seed, scale=0.5):
    rng = np.random.default_rng(seed)
    ps = []
    for l in range(len(dims) - 1):
        ps.append(rng.normal(0, scale / math.sqrt(dims[l]), (dims[l + 1], dims[l])).ravel())
        ps.append(rng.normal(0, 0.1, dims[l + 1]))
    return np.concatenate(ps)


def torch_net(dims, params):
    layers = []
    for W, b in O.mlp_split(dims, params):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(W.copy()))
            lin.bias.copy_(torch.from_numpy(b.copy()))
        layers.append(lin)
    def f(x):
        for i, lin in enumerate(layers):
            x = lin(x)
            if i < len(layers) - 1:
                x = torch.nn.functional.gelu(x, approximate="tanh")
        return x
    return f, layers


def test_gelu_matches_torch_tanh_gelu():
    xs = np.linspace(-8, 8, 321)
    ref = torch.nn.functional.gelu(torch.from_numpy(xs), approximate="tanh").numpy()
    got = np.array([O.gelu(x) for x in xs])
    assert np.max(np.abs(got - ref)) < 1e-14
    # odd part: gelu(x) - gelu(-x) = x
    assert all(abs(O.gelu(x) - O.gelu(-x) - x) < 1e-14 for x in xs)


def test_gelu_grad_matches_autograd_and_differences():
    xs = torch.linspace(-6, 6, 241, dtype=torch.float64, requires_grad=True)
    torch.nn.functional.gelu(xs, approximate="tanh").sum().backward()
    got = np.array([O.gelu_grad(x) for x in xs.detach().numpy()])
    assert np.max(np.abs(got - xs.grad.numpy())) < 1e-13
    h = 1e-6
    fd = np.array([(O.gelu(x + h) - O.gelu(x - h)) / (2 * h) for x in xs.detach().numpy()])
    assert np.max(np.abs(got - fd)) < 1e-8


@pytest.mark.parametrize("dims", [SMALL, O.SUR_DIMS])
def test_forward_matches_torch_layers(dims):
    params = rand_params(dims, 1)
    x = np.random.default_rng(2).uniform(-1, 1, (9, dims[0]))
    f, _ = torch_net(dims, params)
    ref = f(torch.from_numpy(x)).detach().numpy()
    assert np.max(np.abs(O.mlp_forward(dims, params, x) - ref)) < 1e-12


def test_backward_matches_central_differences():
    dims = SMALL
    params = rand_params(dims, 3)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (5, dims[0]))
    dy = rng.normal(0, 1, (5, dims[-1]))
    g = O.mlp_backward(dims, params, x, dy)
    h = 1e-6
    fd = np.zeros_like(params)
    for i in range(params.size):
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd[i] = (np.sum(dy * O.mlp_forward(dims, p1, x)) - np.sum(dy * O.mlp_forward(dims, p2, x))) / (2 * h)
    rel = np.abs(g - fd) / np.maximum(np.abs(fd), 1e-3)
    assert rel.max() < 1e-6


def test_backward_full_width_matches_autograd():
    dims = O.SUR_DIMS
    params = rand_params(dims, 5)
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (4, dims[0]))
    dy = rng.normal(0, 1, (4, dims[-1]))
    g = O.mlp_backward(dims, params, x, dy)
    f, layers = torch_net(dims, params)
    (f(torch.from_numpy(x)) * torch.from_numpy(dy)).sum().backward()
    ref = np.concatenate([t for lin in layers for t in (lin.weight.grad.numpy().ravel(), lin.bias.grad.numpy())])
    assert np.max(np.abs(g - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("stage", [1, 2])
def test_loss_gradient_matches_differences(stage):
    rng = np.random.default_rng(7 + stage)
    y = rng.normal(0, 1, (6, 5))
    t = rng.normal(0, 1, (6, 5))
    mask = np.array([1, 0, 1, 1, 0, 1], dtype=float)
    L, dy = O.sur_loss(stage, y, t, mask)
    h = 1e-7
    for i in range(6):
        for j in range(5):
            y1, y2 = y.copy(), y.copy()
            y1[i, j] += h
            y2[i, j] -= h
            fd = (O.sur_loss(stage, y1, t, mask)[0] - O.sur_loss(stage, y2, t, mask)[0]) / (2 * h)
            assert abs(fd - dy[i, j]) < 1e-7
    # masked samples and the unused outputs of each stage carry no gradient
    assert np.all(dy[mask == 0, :4] == 0) if stage == 1 else np.all(dy[:, :4] == 0)
    assert np.all(dy[:, 4] == 0) if stage == 1 else True
    if stage == 1:
        w = np.array([1, 1, 1, 0.1])
        assert abs(L - np.sum(mask[:, None] * w * (y[:, :4] - t[:, :4]) ** 2) / 6) < 1e-14


def test_adam_matches_torch_optimizer():
    rng = np.random.default_rng(9)
    p = rng.normal(0, 1, 50)
    m, v = np.zeros(50), np.zeros(50)
    tp = torch.nn.Parameter(torch.from_numpy(p.copy()))
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.9, 0.99), eps=1e-8)
    for step in range(1, 8):
        g = rng.normal(0, 1, 50)
        O.adam_step(p, g, m, v, step, lr=3e-3, beta1=0.9, beta2=0.99, eps=1e-8)
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
    assert np.max(np.abs(p - tp.detach().numpy())) < 1e-13


def test_training_set_distribution():
    n = 40000
    R2, H = 1.0, 2.0
    cos_n, z, modes, var = [], [], np.zeros(4), []
    for i in range(n):
        P, d, m, v = O.sur_sample(11, i, R2, H)
        assert abs(math.hypot(P[0], P[1]) - R2) < 1e-15 and abs(P[2]) <= H / 2
        assert abs(np.linalg.norm(d) - 1) < 1e-14
        rh = np.array([P[0], P[1], 0]) / R2
        cos_n.append(-d @ rh)
        z.append(P[2])
        modes[2 * v + m] += 1
    cos_n = np.array(cos_n)
    assert cos_n.min() > 0
    # cosine-weighted hemisphere: E[cos] = 2/3, E[cos^2] = 1/2
    assert abs(cos_n.mean() - 2 / 3) < 0.01 and abs((cos_n ** 2).mean() - 0.5) < 0.01
    assert abs(np.mean(z)) < 0.02 and abs(np.var(z) - H * H / 12) < 0.01
    assert np.all(np.abs(modes / n - 0.25) < 0.01)
    # same seed, same ray; another seed, another ray
    a, b = O.sur_sample(11, 17), O.sur_sample(11, 17)
    assert np.array_equal(a[1], b[1]) and not np.array_equal(a[1], O.sur_sample(12, 17)[1])


def test_features_of_simple_rays():
    P = np.array([0.0, 1.0, 0.5])  # azimuth pi/2, z = 0.5
    a = 0.3
    d = np.array([math.sin(a), -math.cos(a), 0.0])  # theta-hat at pi/2 is (-1, 0, 0): d_theta = -sin(a)
    x = O.sur_features(0.5, 1.0, 2.0, 1, 0, P, d)
    assert np.allclose(x, [0.5, -0.5, 0.0, -a / (math.pi / 2), -1.0, 1.0, 0.5], atol=1e-15)
    d2 = np.array([0.0, -math.cos(a), math.sin(a)])
    x2 = O.sur_features(0.5, 1.0, 2.0, 0, 1, P, d2)
    assert abs(x2[2] - a / (math.pi / 2)) < 1e-15 and abs(x2[3]) < 1e-15


def _traced_training_rays(n, seed, integ):
    R1, R2, H = 0.5, 1.0, 2.0
    out = []
    for i in range(n):
        P, d, m, v = O.sur_sample(seed, i, R2, H)
        o = P - 0.5 * d
        rec, _ = O.trace_ray(O.Cloak(v, R1, R2, H), integ, m, o, d)
        out.append((P, d, m, v, rec))
    return out


def test_targets_reconstruct_traced_rays():
    """Conservation of k_z and L_z: the exit of every laterally exiting ray is rebuilt from its exit
    azimuth, height and time of flight alone."""
    integ = O.Integrator(O.DP45, 1e-10, 2_000_000)
    n_lat = 0
    for P, d, m, v, rec in _traced_training_rays(120, 21, integ):
        ok, t = O.sur_targets(1.0, 2.0, P, d, rec)
        if not ok:
            assert rec["status"] not in (1, 2) or abs(abs(rec["exit_pos"][2]) - 1.0) < 1e-9
            continue
        n_lat += 1
        pos, dr, tof = O.sur_reconstruct(1.0, 2.0, P, d, t)
        assert np.max(np.abs(pos - rec["exit_pos"])) < 1e-12
        assert np.max(np.abs(dr - rec["exit_dir"])) < 1e-7
        assert abs(tof - rec["tof"]) < 1e-14
        assert abs(t[1] ** 2 + t[2] ** 2 - 1) < 1e-14
    assert n_lat > 40


def test_targets_do_not_depend_on_entry_height_or_azimuth():
    """Translation and rotation symmetry of both media: the same direction in the local frame at another
    entry height and azimuth gives the same targets (while the exit stays lateral)."""
    integ = O.Integrator(O.DP45, 1e-11, 2_000_000)
    for variant, mode in ((O.RADIAL, O.EXTRAORDINARY), (O.AZIMUTHAL, O.ORDINARY), (O.AZIMUTHAL, O.EXTRAORDINARY)):
        ts = []
        for phi, z in ((0.3, -0.2), (2.5, 0.15), (4.4, 0.0)):
            rh, th = np.array([math.cos(phi), math.sin(phi), 0]), np.array([-math.sin(phi), math.cos(phi), 0])
            d = -0.8 * rh + 0.5 * th + math.sqrt(1 - 0.64 - 0.25) * np.array([0, 0, 1.0])
            P = rh + np.array([0, 0, z])
            rec, _ = O.trace_ray(O.Cloak(variant), integ, mode, P - 0.5 * d, d)
            ok, t = O.sur_targets(1.0, 2.0, P, d, rec)
            assert ok
            ts.append(t)
        assert np.max(np.abs(np.array(ts) - ts[0])) < 1e-8, (variant, mode, ts)


def test_in_plane_extraordinary_rays_follow_the_straight_line():
    """Perfect cloaking for in-plane rays (Eq. 13 matching): psi = 0, exit height = entry height,
    time of flight = vacuum chord, for both cloaks."""
    integ = O.Integrator(O.DP45, 1e-11, 2_000_000)
    for variant in (O.RADIAL, O.AZIMUTHAL):
        for beta in (-1.2, -0.4, 0.25, 0.9):
            phi = 0.7
            P = np.array([math.cos(phi), math.sin(phi), 0.1])
            rh, th = np.array([math.cos(phi), math.sin(phi), 0]), np.array([-math.sin(phi), math.cos(phi), 0])
            d = -math.cos(beta) * rh + math.sin(beta) * th
            rec, _ = O.trace_ray(O.Cloak(variant), integ, O.EXTRAORDINARY, P - 0.5 * d, d)
            ok, t = O.sur_targets(1.0, 2.0, P, d, rec)
            assert ok
            assert abs(t[0]) < 1e-9 and abs(t[2]) < 1e-8 and abs(t[1] - 1) < 1e-12
            assert abs(4 * t[3] - 2 * math.cos(beta)) < 1e-8
