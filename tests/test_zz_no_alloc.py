"""Allocation-free render: cloak_render_noalloc against cloak_render.

Some callers may not allocate device memory -- their device memory belongs to another allocator, or
the device-wide synchronisation of cudaMalloc / cudaFree is not acceptable inside their render loop.
For them the library renders from one fixed device array that it owns (at most 1048576 samples per
call).  Through the C ABI, this file checks that two calls in a row give the images that
cloak_render gives for the same settings (the second call starts from the first call's leftover
contents), and that a size beyond the array's limit is refused before any launch.

The file name sorts last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1209_6038_gb300 import inputs

pytestmark = pytest.mark.gpu

IMAGE_TOL = 1e-5  # the image tolerance of the parity tests


@pytest.fixture(scope="module")
def ck():
    import torch
    from paper_1209_6038_gb300 import build, cloak
    build.build()
    cloak.load()
    torch.cuda.init()
    return cloak


def reference_and_noalloc(ck, variant, mode, elev, W, H, spp, seed, precision):
    import torch
    eye, tgt, up = inputs.camera_pose(elev)
    c = ck.Cloak(variant).camera(eye, tgt, up, 60.0, W, H).integrator(ck.DP45, 1e-9, precision)
    c.schedule(ck.SCHED_WAVEFRONT)
    ref = c.render(mode, spp, seed)
    out = torch.full((H, W, 4), -1.0, dtype=torch.float32, device="cuda")
    ck.cloak_render_noalloc(c.h, mode, spp, seed, out)
    torch.cuda.synchronize()
    c.close()
    return ref.cpu().numpy(), out.cpu().numpy()


def test_noalloc_two_calls_match_render(ck):
    # call 1: azimuthal cloak, extraordinary light, 320x180 x 4 spp, FP64
    ref, got = reference_and_noalloc(ck, 1, 1, 20.0, 320, 180, 4, 11, ck.FP64)
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= IMAGE_TOL
    # call 2 (leftover contents of call 1 in the array): radial cloak, ordinary light,
    # 512x512 x 4 spp = exactly the 1048576-sample limit, mixed precision
    ref, got = reference_and_noalloc(ck, 0, 0, 45.0, 512, 512, 4, 12, ck.MIXED)
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= IMAGE_TOL


def test_noalloc_rejects_oversize(ck):
    import torch
    c = ck.Cloak(0).camera((5, 0, 0), (0, 0, 0), (0, 0, 1), 60.0, 513, 512).integrator(ck.DP45, 1e-9)
    out = torch.zeros((512, 513, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(ck.CloakError) as ei:
        ck.cloak_render_noalloc(c.h, 1, 4, 0, out)
    assert ei.value.code == ck.EINVAL
    assert "no-alloc limit" in str(ei.value)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0  # nothing was launched
    c.close()
