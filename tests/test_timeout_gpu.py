"""Failure detection on the GPU without a fault: the bounded waits of the tensor-core kernels.

cloak_set_wait_limit(1) lowers the poll bound of the waits that decide a timeout to one non-blocking poll,
so the first wait for a TMA copy runs out on an ordinary launch.  The kernel must report it (the flag ->
CLOAK_ETIMEOUT), let its in-flight copies and MMAs land, free its TMEM and leave the context usable: the
next call with the default bound succeeds and is correct.  A CLOAK_SURROGATE render whose network timed out
must leave every ray to the FP64 integrator, so its image equals the integrator's."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture
def ck():
    from paper_1209_6038_gb300 import cloak
    cloak.load()
    yield cloak
    cloak.cloak_set_wait_limit(0)  # the default bound for every later test


def test_gemm_wait_runs_out_then_recovers(ck):
    M, N, K = 1024, 256, 4096
    g = torch.Generator(device="cuda").manual_seed(0)
    a = torch.randn(M, K, device="cuda", generator=g).bfloat16()
    b = torch.randn(N, K, device="cuda", generator=g).bfloat16()
    c = torch.zeros(M, N, device="cuda")
    ck.cloak_set_wait_limit(1)
    for _ in range(2):  # twice: the first timeout left nothing behind that blocks the second launch
        with pytest.raises(ck.CloakError) as ei:
            ck.cloak_mlp_gemm(a, b, c)
        assert ei.value.code == ck.ETIMEOUT
    ck.cloak_set_wait_limit(0)
    ck.cloak_mlp_gemm(a, b, c)
    ref = a.float() @ b.float().T
    assert torch.allclose(c, ref, rtol=1e-3, atol=2e-2)


def test_wait_limit_rejects_bad_values(ck):
    with pytest.raises(ck.CloakError) as ei:
        ck.cloak_set_wait_limit(-1)
    assert ei.value.code == ck.EINVAL
    with pytest.raises(ck.CloakError):
        ck.cloak_set_wait_limit(1 << 33)


def test_surrogate_forward_times_out_then_recovers(ck):
    c = ck.Cloak(ck.RADIAL)
    ck.cloak_surrogate_params(c.h, ck.cloak_surrogate_params(c.h))  # seeded initial weights
    n = 4096
    x = torch.rand((n, 7), device="cuda", generator=torch.Generator(device="cuda").manual_seed(1)) * 2 - 1
    y0 = torch.empty((n, 5), device="cuda")
    ck.cloak_surrogate_forward(c.h, x, y0)
    ck.cloak_set_wait_limit(1)
    y1 = torch.full((n, 5), 7.0, device="cuda")
    with pytest.raises(ck.CloakError) as ei:
        ck.cloak_surrogate_forward(c.h, x, y1)
    assert ei.value.code == ck.ETIMEOUT
    ck.cloak_set_wait_limit(0)
    ck.cloak_surrogate_forward(c.h, x, y1)
    assert torch.equal(y0, y1)
    c.close()


def test_surrogate_render_falls_back_to_the_integrator_on_timeout(ck):
    from paper_1209_6038_gb300 import inputs
    W, H = 96, 64
    eye, tgt, up = inputs.camera_pose(0.0)
    c = ck.Cloak(ck.RADIAL).camera(eye, tgt, up, 60.0, W, H).schedule(ck.SCHED_WAVEFRONT)
    c.integrator(ck.DP45, 1e-9, ck.FP64)
    ck.cloak_surrogate_train(c.h, 2 * 19456, seed=3, epochs=1)
    ref = c.render(ck.POL_EXTRAORDINARY, spp=2, seed=0)
    views_ref = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
    vlist = lambda outs: [(v, ck.POL_EXTRAORDINARY, eye, tgt, up, 60.0, o) for v, o in zip((ck.RADIAL, ck.RADIAL), outs)]
    ck.cloak_render_batch(c.h, vlist(views_ref), 2, 0)
    # a network whose last layer is constant: exit height = entry height, exit azimuth on the straight line,
    # predicted log10 error -20 -- the gate takes every ray in its support, and the images differ
    params = ck.cloak_surrogate_params(c.h)
    params[-5 - 5 * 256:] = 0.0
    params[-5:] = [0.0, 1.0, 0.0, 0.5, -20.0]
    ck.cloak_surrogate_params(c.h, params)
    c.integrator(ck.DP45, 1e-9, ck.SURROGATE)
    sur = c.render(ck.POL_EXTRAORDINARY, spp=2, seed=0)
    torch.cuda.synchronize()
    assert not torch.equal(sur, ref)
    ck.cloak_set_wait_limit(1)
    fb = c.render(ck.POL_EXTRAORDINARY, spp=2, seed=0)
    views_fb = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
    ck.cloak_render_batch(c.h, vlist(views_fb), 2, 0)
    torch.cuda.synchronize()
    ck.cloak_set_wait_limit(0)
    assert torch.equal(fb, ref)
    for a, b in zip(views_fb, views_ref):
        assert torch.equal(a, b)
    # the default bound again: the network's exits are used once more (the captured graph was re-made)
    views_sur = [torch.empty((H, W, 4), device="cuda") for _ in range(2)]
    ck.cloak_render_batch(c.h, vlist(views_sur), 2, 0)
    torch.cuda.synchronize()
    assert not torch.equal(views_sur[0], views_ref[0])
    c.close()
