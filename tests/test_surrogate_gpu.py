"""Learned surrogate on the GPU (tcgen05 BF16 forward / backward, Adam, gate) against the FP64 oracle of
oracle/surrogate_oracle.c, and what it gains over the integrator alone."""
import math
import os
import time

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

DIMS = O.SUR_DIMS
BF16_U = 2.0 ** -9  # unit roundoff of BF16 (8 significant bits)
F16_U = 2.0 ** -11  # unit roundoff of FP16 (11 significant bits)


@pytest.fixture(scope="module")
def ck():
    import torch
    from paper_1209_6038_gb300 import build, cloak
    build.build()
    cloak.load()
    torch.cuda.init()
    return cloak


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def init_params(seed, out_scale=0.1):
    rng = np.random.default_rng(seed)
    ps = []
    for l in range(len(DIMS) - 1):
        sd = (out_scale if l == len(DIMS) - 2 else 1.0) / math.sqrt(DIMS[l])
        ps.append(rng.normal(0, sd, (DIMS[l + 1], DIMS[l])).ravel())
        ps.append(rng.normal(0, 0.05, DIMS[l + 1]))
    return np.concatenate(ps).astype(np.float32)


def bf16_weights(params):
    """The network the tensor cores evaluate: weights rounded to BF16, biases FP32."""
    out = params.astype(np.float64).copy()
    o = 0
    for l in range(len(DIMS) - 1):
        nw = DIMS[l + 1] * DIMS[l]
        out[o:o + nw] = bf16(out[o:o + nw])
        o += nw + DIMS[l + 1]
    return out


def f16_inference_params(params):
    """The network the fused inference kernel evaluates: weights rounded to FP16, the hidden layers' biases
    rounded to FP16, the output layer's biases FP32."""
    out = params.astype(np.float64).copy()
    o = 0
    for l in range(len(DIMS) - 1):
        nw, nb = DIMS[l + 1] * DIMS[l], DIMS[l + 1]
        out[o:o + nw] = out[o:o + nw].astype(np.float32).astype(np.float16).astype(np.float64)
        if l < len(DIMS) - 2:
            out[o + nw:o + nw + nb] = out[o + nw:o + nw + nb].astype(np.float32).astype(np.float16).astype(np.float64)
        o += nw + nb
    return out


def layer_slices():
    sl, o = [], 0
    for l in range(len(DIMS) - 1):
        nw = DIMS[l + 1] * DIMS[l]
        sl.append((slice(o, o + nw), slice(o + nw, o + nw + DIMS[l + 1])))
        o += nw + DIMS[l + 1]
    return sl


def make_handle(ck, params):
    h = ck.Cloak(ck.RADIAL)
    ck.cloak_surrogate_params(h.h, params)
    return h


@pytest.mark.parametrize("fp16", [False, True])
def test_forward_matches_oracle(ck, fp16):
    import torch
    params = init_params(1, out_scale=1.0)
    h = make_handle(ck, params)
    ck.cloak_surrogate_set_precision(h.h, fp16)
    rng = np.random.default_rng(2)
    n = 1000
    x = rng.uniform(-1, 1, (n, 7)).astype(np.float32)
    y = torch.zeros((n, 5), dtype=torch.float32, device="cuda")
    ck.cloak_surrogate_forward(h.h, torch.from_numpy(x).cuda(), y)
    got = y.cpu().numpy().astype(np.float64)
    scale_u = F16_U if fp16 else BF16_U
    ref = O.mlp_forward(DIMS, f16_inference_params(params) if fp16 else bf16_weights(params), x.astype(np.float64))
    # BF16 (default): weights rounded to BF16 as the reference has them, inputs as BF16 (hi, lo) pairs
    # (about 16 bits), each of the 4 hidden activations rounded to BF16 (relative error <= 2^-9), FP32
    # accumulation.  FP16: weights and hidden biases rounded to FP16 (the reference uses the same values),
    # inputs as FP16 pairs (about 22 bits), activations rounded to FP16 (2^-11).  The GELU runs in
    # half-precision pairs in both (hardware tanh, relative error ~2^-11).  With unit-gain layers the output
    # error stays within a few units of the activations' unit roundoff times the output scale.
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max()
    print(f"forward error ({'FP16' if fp16 else 'BF16'}) {err / scale / scale_u:.2f} units roundoff of the output scale")
    assert err <= 8 * scale_u * scale, (err, scale)
    assert np.isfinite(got).all()
    h.close()


def _batch(n, seed, stage):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, (n, 7)).astype(np.float32)
    t = np.zeros((n, 8), np.float32)
    t[:, :5] = rng.normal(0, 1, (n, 5))
    t[:, 5] = (rng.uniform(0, 1, n) < 0.8)
    return x, t


@pytest.mark.parametrize("stage,n", [(1, 256), (2, 256), (1, 19456), (2, 4864)])
def test_gradients_match_oracle(ck, stage, n):
    """n = 256: each weight-gradient GEMM splits the batch into 4 slices of one 64-row chunk; 4864 and 19456
    (the training batch): 76 or 152 slices of one or several chunks each, summed in a fixed order."""
    import torch
    params = init_params(3, out_scale=1.0)
    h = make_handle(ck, params)
    x, t = _batch(n, 4 + stage, stage)
    g = ck.cloak_surrogate_step(h.h, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), stage=stage, lr=0.0)
    W = bf16_weights(params)
    xb = x.astype(np.float64)
    y = O.mlp_forward(DIMS, W, xb)
    _, dy = O.sur_loss(stage, y, t[:, :5], t[:, 5])
    ref = O.mlp_backward(DIMS, W, xb, dy)
    # BF16 rounding of activations, of dL/dY and of every back-propagated dZ: relative error of a
    # layer's gradient a few percent at most; the direction must agree closely
    for l, (sw, sb) in enumerate(layer_slices()):
        for s in (sw, sb):
            a, b = g[s].astype(np.float64), ref[s]
            nb = np.linalg.norm(b)
            if nb == 0:
                assert np.linalg.norm(a) == 0
                continue
            rel = np.linalg.norm(a - b) / nb
            cos = a @ b / (np.linalg.norm(a) * nb)
            assert rel < 0.05 and cos > 0.998, (stage, l, rel, cos)
    h.close()


def test_adam_step_matches_oracle(ck):
    import torch
    params = init_params(7)
    h = make_handle(ck, params)
    n = 384
    x, t = _batch(n, 8, 1)
    lr = 1e-3
    g = ck.cloak_surrogate_step(h.h, torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), stage=1, lr=lr)
    new = ck.cloak_surrogate_params(h.h)
    p = params.astype(np.float64).copy()
    m, v = np.zeros_like(p), np.zeros_like(p)
    O.adam_step(p, g.astype(np.float64), m, v, 1, lr=lr, beta1=0.9, beta2=0.999, eps=1e-8)
    # the weights of the entry height and azimuth (first layer, inputs 0 and 1) are not trained
    frozen = (np.arange(DIMS[1])[:, None] * DIMS[0] + np.array([0, 1])[None, :]).ravel()
    p[frozen] = params[frozen]
    # same gradient, FP32 update arithmetic against FP64
    assert np.max(np.abs(new - p)) <= 1e-6 * max(1.0, np.abs(p).max())
    assert np.max(np.abs(new - params)) > 0.5 * lr
    h.close()


def test_checkpoint_round_trip(ck, tmp_path):
    import torch
    params = init_params(9, out_scale=1.0)
    h = make_handle(ck, params)
    x = torch.rand((300, 7), device="cuda") * 2 - 1
    y1 = torch.zeros((300, 5), device="cuda")
    ck.cloak_surrogate_forward(h.h, x, y1)
    path = str(tmp_path / "sur.bin")
    ck.cloak_surrogate_save(h.h, path)
    h2 = ck.Cloak(ck.RADIAL)
    ck.cloak_surrogate_load(h2.h, path)
    y2 = torch.zeros_like(y1)
    ck.cloak_surrogate_forward(h2.h, x, y2)
    assert torch.equal(y1, y2)
    assert np.array_equal(ck.cloak_surrogate_params(h2.h), params)
    with open(path, "r+b") as f:
        f.write(b"XXXXXXXX")
    with pytest.raises(ck.CloakError):
        ck.cloak_surrogate_load(h2.h, path)
    h.close()
    h2.close()


@pytest.fixture(scope="module")
def trained(ck):
    """A surrogate trained on 2^21 rays traced by the FP64 DP5(4) integrator at tolerance 1e-9."""
    h = ck.Cloak(ck.RADIAL).integrator(ck.DP45, 1e-9, ck.FP64, 1_000_000)
    t0 = time.perf_counter()
    ck.cloak_surrogate_train(h.h, 1 << 21, seed=11, epochs=40)
    info = ck.cloak_surrogate_info(h.h)
    info["wall"] = time.perf_counter() - t0
    yield h, info
    h.close()


def test_training_converges(ck, trained):
    h, info = trained
    print(info)
    assert info["rays"] == 1 << 21
    assert 0.3 < info["lateral_fraction"] < 1.0
    assert info["loss_stage1"] < 3e-4, info
    assert math.isfinite(info["loss_stage2"])


def _handles(ck, trained_h, variant, elev, W, H, precision):
    from paper_1209_6038_gb300 import inputs
    eye, tgt, up = inputs.camera_pose(elev)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, precision, 1_000_000)
    c.schedule(ck.SCHED_WAVEFRONT)
    return c


@pytest.mark.parametrize("variant,mode,elev,fp16", [(0, 1, 20.0, False), (1, 1, 0.0, False), (1, 0, 45.0, False),
                                                    (0, 0, 20.0, False), (0, 1, 20.0, True), (1, 1, 0.0, True)])
def test_surrogate_records_keep_invariants_and_match_oracle(ck, trained, tmp_path, variant, mode, elev, fp16):
    """Rays finished by the surrogate leave through r = R2 with k_z and L_z of the camera ray (exact), and
    their exit direction agrees with the FP64 oracle within the gate; all other rays are the integrator's.
    Inference in BF16 (the default) and in FP16."""
    import torch
    from paper_1209_6038_gb300 import inputs
    h, _ = trained
    path = str(tmp_path / "s.bin")
    ck.cloak_surrogate_save(h.h, path)
    W, H = 96, 54
    c = _handles(ck, h, variant, elev, W, H, ck.SURROGATE)
    ck.cloak_surrogate_load(c.h, path)
    ck.cloak_surrogate_set_precision(c.h, fp16)
    ck.cloak_surrogate_set_gate(c.h, -2.5)
    recs = ck.records_to_numpy(c.render_records(mode, 1, 0))
    ref = _handles(ck, h, variant, elev, W, H, ck.FP64)
    rref = ck.records_to_numpy(ref.render_records(mode, 1, 0))
    sur = (recs["steps"] == 0) & np.isin(recs["status"], [1, 2])
    assert sur.sum() > 0
    # the metal flag of radial o-rays is exact geometry (straight lines inside)
    assert (recs["status"][sur] == rref["status"][sur]).mean() >= 0.99
    # integrator rays are bit-identical to the FP64 render
    rest = ~sur
    for f in ("exit_pos", "exit_dir", "tof", "weight", "tile_id", "status", "steps"):
        assert np.array_equal(recs[f][rest], rref[f][rest]), f
    # exact invariants of the surrogate's exit (camera rays of a pinhole at eye, one sample per pixel)
    eye, tgt, up = inputs.camera_pose(elev)
    cam = O.Camera(eye, tgt, up, 60.0, W, H)
    idx = np.nonzero(sur)[0]
    for k in idx[:: max(1, len(idx) // 200)]:
        o, d = O.camera_ray(cam, k % W, k // W, 0, 1, 0)
        pe, de = recs["exit_pos"][k], recs["exit_dir"][k]
        assert abs(math.hypot(pe[0], pe[1]) - 1.0) < 1e-12
        assert abs(de[2] - d[2]) < 1e-12
        assert abs((pe[0] * de[1] - pe[1] * de[0]) - (o[0] * d[1] - o[1] * d[0])) < 1e-11
    # against the FP64 oracle: the gate keeps the exit error small for the rays it lets through
    cl = O.Cloak(variant)
    integ = O.Integrator(O.DP45, 1e-9, 1_000_000)
    errs = []
    for k in idx[:: max(1, len(idx) // 150)]:
        o, d = O.camera_ray(cam, k % W, k // W, 0, 1, 0)
        r, _ = O.trace_ray(cl, integ, mode, o, d)
        a, b = recs["exit_dir"][k], r["exit_dir"]
        errs.append(math.atan2(np.linalg.norm(np.cross(a, b)), a @ b))
    errs = np.array(errs)
    print(variant, mode, elev, "handled", sur.sum(), "median", np.median(errs), "p90", np.quantile(errs, 0.9), "max", errs.max())
    assert np.median(errs) < 3e-3 and np.quantile(errs, 0.9) < 1e-2, (np.median(errs), errs.max())
    c.close()
    ref.close()


def test_surrogate_gains_over_the_integrator(ck, trained, tmp_path):
    """The surrogate with integrator fallback renders faster than the integrator alone, at a stated image
    error: most cloak pixels keep their room tile."""
    import torch
    h, _ = trained
    path = str(tmp_path / "s.bin")
    ck.cloak_surrogate_save(h.h, path)
    W, H = 640, 360
    res = {}
    for name, prec in (("fp64", ck.FP64), ("surrogate", ck.SURROGATE)):
        c = _handles(ck, h, 1, 20.0, W, H, prec)
        if prec == ck.SURROGATE:
            ck.cloak_surrogate_load(c.h, path)
            ck.cloak_surrogate_set_gate(c.h, -3.0)
        out = torch.empty((H, W, 4), device="cuda")
        c.render(1, 1, 0, out=out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            c.render(1, 1, 0, out=out)
        torch.cuda.synchronize()
        res[name] = ((time.perf_counter() - t0) / 3, c.render_records(1, 1, 0))
        c.close()
    t64, r64 = res["fp64"]
    tsu, rsu = res["surrogate"]
    a, b = ck.records_to_numpy(r64), ck.records_to_numpy(rsu)
    entering = a["status"] != 0
    tile_diff = (a["tile_id"] != b["tile_id"]) & entering
    frac = tile_diff.sum() / max(1, entering.sum())
    handled = ((b["steps"] == 0) & np.isin(b["status"], [1, 2])).sum() / max(1, entering.sum())
    print(f"fp64 {t64 * 1e3:.1f} ms, surrogate {tsu * 1e3:.1f} ms, handled {handled:.3f}, tile differs {frac:.4f}")
    # stated image error at gate -3: fewer than 5 % of the cloak's pixels see another room tile (the share
    # the gate passes varies between training runs: 20-50 % of the entering rays for this training set)
    assert handled > 0.1
    assert frac < 0.05
    assert tsu < t64


@pytest.mark.parametrize("fp16", [False, True])
def test_batched_surrogate_render_matches_single_renders(ck, trained, tmp_path, fp16):
    """The learned surrogate inside the batched persistent render (one queue for all views, the network and
    gate on every queued ray, the integrator on the rest): each view equals its own surrogate render, with
    the network in BF16 (default) and in FP16."""
    import torch
    h, _ = trained
    path = str(tmp_path / "s.bin")
    ck.cloak_surrogate_save(h.h, path)
    views, refs = [], []
    for variant, pol, elev, W, H in ((1, 1, 20.0, 96, 64), (0, 0, 0.0, 80, 48), (1, 0, 45.0, 64, 64), (0, 1, 10.0, 72, 40)):
        c = _handles(ck, h, variant, elev, W, H, ck.SURROGATE)
        ck.cloak_surrogate_load(c.h, path)
        ck.cloak_surrogate_set_precision(c.h, fp16)
        ck.cloak_surrogate_set_gate(c.h, -3.0)
        refs.append(c.render(pol, 2, 4).cpu().numpy())
        from paper_1209_6038_gb300 import inputs
        eye, tgt, up = inputs.camera_pose(elev)  # the pose of _handles
        views.append((variant, pol, eye, tgt, up, 60.0, torch.empty((H, W, 4), device="cuda")))
        c.close()
    b = ck.Cloak(ck.RADIAL).integrator(ck.DP45, 1e-9, ck.SURROGATE, 1_000_000).schedule(ck.SCHED_WAVEFRONT)
    ck.cloak_surrogate_load(b.h, path)
    ck.cloak_surrogate_set_precision(b.h, fp16)
    ck.cloak_surrogate_set_gate(b.h, -3.0)
    for _ in range(2):  # capture, then replay of the graph
        ck.cloak_render_batch(b.h, views, 2, 4)
        torch.cuda.synchronize()
        for (_, _, _, _, _, _, out), ref in zip(views, refs):
            assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-6
    b.close()


def test_training_is_reproducible_and_timed(ck):
    """The same seed trains the same network bit for bit: the weight gradients of the batch-split GEMMs are
    summed in a fixed order (no atomics).  The training reports its device time per optimizer step."""
    nets = []
    for _ in range(2):
        c = ck.Cloak(ck.RADIAL).integrator(ck.DP45, 1e-9, ck.FP64)
        ck.cloak_surrogate_train(c.h, 3 * 19456, seed=21, epochs=3)
        nets.append(ck.cloak_surrogate_params(c.h))
        t = ck.cloak_surrogate_train_timing(c.h)
        assert t["ms_per_step_stage1"] > 0 and t["ms_per_step_stage2"] > 0 and t["batch"] == 19456
        assert t["flops_per_step_stage1"] == pytest.approx(2 * 19456 * (2 * 199680 + 197888))
        c.close()
    assert np.array_equal(nets[0], nets[1])
    c = ck.Cloak(ck.RADIAL)
    with pytest.raises(ck.CloakError):
        ck.cloak_surrogate_train_timing(c.h)
    c.close()
