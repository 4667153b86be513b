"""Thin Python binding of the C ABI in include/cloak.h (argument marshalling only).

The functions carry the C names; every step of the rendering path runs in the
CUDA kernels of libcloak.so.  Device buffers are torch tensors; the current
torch stream is passed as the CUDA stream.  Loading fails loudly when the
library has not been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcloak.so")

RADIAL, AZIMUTHAL, TEST_UNIAXIAL_CONST = 0, 1, 100
POL_ORDINARY, POL_EXTRAORDINARY = 0, 1
RK4, DP45 = 0, 1
FP64, MIXED, MIXED_FF, SURROGATE = 0, 1, 2, 3
SCHED_PLAIN, SCHED_WAVEFRONT = 0, 1
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = range(6)
RAY_STATUS = {0: "MISSED", 1: "EXITED", 2: "HIT_METAL_EXITED", 3: "NO_TRANSMISSION", 4: "TIR",
              5: "STEP_LIMIT", 6: "SINGULAR", 7: "METAL_CAP"}

RECORD_DTYPE = np.dtype([("exit_pos", "<f8", 3), ("exit_dir", "<f8", 3), ("tof", "<f8"), ("weight", "<f8"),
                         ("tile_id", "<i4"), ("status", "<i4"), ("steps", "<i4"), ("mode", "<i4")])
RECORD_BYTES = 80

# name -> (restype, argtypes) of every entry point declared in include/cloak.h
_d3 = C.POINTER(C.c_double)
SIGNATURES = {
    "cloak_create": (C.c_void_p, [C.c_int, C.c_double, C.c_double, C.c_double]),
    "cloak_destroy": (None, [C.c_void_p]),
    "cloak_last_error": (C.c_char_p, []),
    "cloak_camera_set": (C.c_int, [C.c_void_p, _d3, _d3, _d3, C.c_double, C.c_int, C.c_int]),
    "cloak_set_integrator": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_long]),
    "cloak_set_test_medium": (C.c_int, [C.c_void_p, C.c_double, C.c_double, _d3]),
    "cloak_set_scene_seed": (C.c_int, [C.c_void_p, C.c_ulonglong]),
    "cloak_set_schedule": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "cloak_set_stage_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "cloak_set_schedule_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double]),
    "cloak_stage_times": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "cloak_render": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p, C.c_size_t, C.c_void_p]),
    "cloak_render_records": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p, C.c_size_t,
                                       C.c_void_p]),
    "cloak_trace_rays": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_long, C.c_void_p, C.c_void_p]),
    "cloak_eval_rhs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_long, C.c_void_p, C.c_void_p]),
    "cloak_mlp_gemm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "cloak_set_wait_limit": (C.c_int, [C.c_longlong]),
    "cloak_fma_peak": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_longlong, C.c_void_p, C.POINTER(C.c_double),
                                 C.c_void_p]),
    "cloak_render_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p]),
    "cloak_render_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p, C.c_size_t,
                                       C.c_void_p]),
    "cloak_set_analyzer": (C.c_int, [C.c_void_p, C.c_int]),
    "cloak_set_reflections": (C.c_int, [C.c_void_p, C.c_int]),
    "cloak_set_formulation": (C.c_int, [C.c_void_p, C.c_int]),
    "cloak_render_panel": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_ulonglong, C.c_void_p, C.c_size_t,
                                     C.c_void_p]),
    "cloak_surrogate_train": (C.c_int, [C.c_void_p, C.c_long, C.c_ulonglong, C.c_int, C.c_void_p]),
    "cloak_surrogate_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "cloak_surrogate_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "cloak_surrogate_set_gate": (C.c_int, [C.c_void_p, C.c_double]),
    "cloak_surrogate_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "cloak_surrogate_set_precision": (C.c_int, [C.c_void_p, C.c_int]),
    "cloak_surrogate_train_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "cloak_surrogate_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_long, C.c_int]),
    "cloak_surrogate_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_long, C.c_void_p, C.c_void_p]),
    "cloak_surrogate_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_long, C.c_int, C.c_double,
                                       C.POINTER(C.c_float), C.c_void_p]),
}

class View(C.Structure):
    """cloak_view of include/cloak.h"""
    _fields_ = [("variant", C.c_int), ("polarization", C.c_int), ("eye", C.c_double * 3), ("target", C.c_double * 3),
                ("up", C.c_double * 3), ("hfov_deg", C.c_double), ("width", C.c_int), ("height", C.c_int),
                ("dev_rgba", C.c_void_p)]


_lib = None


class CloakError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cloak error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    """Load libcloak.so and declare the signatures.  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; "
                               "g.build()'); there is no CPU fallback")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc):
    if rc != OK:
        raise CloakError(rc, load().cloak_last_error().decode())
    return rc


def _vec3(v):
    return (C.c_double * 3)(*[float(x) for x in v])


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ C names
def cloak_create(variant, R1, R2, height):
    h = load().cloak_create(variant, R1, R2, height)
    if not h:
        raise CloakError(EINVAL, load().cloak_last_error().decode())
    return C.c_void_p(h)


def cloak_destroy(h):
    load().cloak_destroy(h)


def cloak_last_error():
    return load().cloak_last_error().decode()


def cloak_camera_set(h, eye, target, up, hfov_deg, width, height):
    return _check(load().cloak_camera_set(h, _vec3(eye), _vec3(target), _vec3(up), hfov_deg, width, height))


def cloak_set_integrator(h, kind, h_or_tol, precision=FP64, max_steps=1_000_000):
    return _check(load().cloak_set_integrator(h, kind, h_or_tol, precision, max_steps))


def cloak_set_test_medium(h, eps_o, eps_e, c_hat):
    return _check(load().cloak_set_test_medium(h, eps_o, eps_e, _vec3(c_hat)))


def cloak_set_scene_seed(h, seed):
    return _check(load().cloak_set_scene_seed(h, seed))


def cloak_set_schedule(h, schedule, packet=0, steps_per_round=0):
    return _check(load().cloak_set_schedule(h, schedule, packet, steps_per_round))


def cloak_set_schedule_tuning(h, long_ray_blocks=4, reserve_per_thread=1, cost_scale=4.0):
    return _check(load().cloak_set_schedule_tuning(h, long_ray_blocks, reserve_per_thread, cost_scale))


def cloak_set_stage_timing(h, on):
    return _check(load().cloak_set_stage_timing(h, 1 if on else 0))


def cloak_stage_times(h):
    """[camera+entry, integration, exit+shading, resolve] of the last render, in ms."""
    ms = (C.c_float * 4)()
    _check(load().cloak_stage_times(h, ms))
    return list(ms)


def cloak_render(h, polarization, spp, seed, rgba, stream=None):
    """rgba: float32 CUDA tensor with >= 4*W*H elements."""
    return _check(load().cloak_render(h, polarization, spp, seed, C.c_void_p(rgba.data_ptr()),
                                      rgba.numel() * rgba.element_size(), _stream_ptr(stream)))


def cloak_render_records(h, polarization, spp, seed, records, stream=None):
    """records: uint8 (or any) CUDA tensor of >= 80*W*H*spp bytes."""
    return _check(load().cloak_render_records(h, polarization, spp, seed, C.c_void_p(records.data_ptr()),
                                              records.numel() * records.element_size(), _stream_ptr(stream)))


def cloak_trace_rays(h, polarization, rays, n, records, stream=None):
    """rays: float64 CUDA tensor (n, 6); records: CUDA tensor of >= 80*n bytes."""
    if records.numel() * records.element_size() < RECORD_BYTES * n or rays.numel() < 6 * n:
        raise CloakError(EINVAL, "buffer too small")
    return _check(load().cloak_trace_rays(h, polarization, C.c_void_p(rays.data_ptr()), n,
                                          C.c_void_p(records.data_ptr()), _stream_ptr(stream)))


def cloak_eval_rhs(h, polarization, y, n, dy, stream=None):
    """y, dy: float64 CUDA tensors of >= 6*n elements (states and their derivatives)."""
    if y.numel() < 6 * n or dy.numel() < 6 * n:
        raise CloakError(EINVAL, "buffer too small")
    return _check(load().cloak_eval_rhs(h, polarization, C.c_void_p(y.data_ptr()), n, C.c_void_p(dy.data_ptr()),
                                        _stream_ptr(stream)))


def cloak_mlp_gemm(a, b, c, stream=None):
    """c[M, N] (fp32) = a[M, K] (bf16) @ b[N, K]^T (bf16) on the tensor cores."""
    M, K = a.shape
    N = b.shape[0]
    return _check(load().cloak_mlp_gemm(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(c.data_ptr()),
                                        M, N, K, _stream_ptr(stream)))


def cloak_set_wait_limit(polls=0):
    """Polls of the tensor-core kernels' bounded waits (0: the default 2^22)."""
    return _check(load().cloak_set_wait_limit(int(polls)))


def cloak_fma_peak(precision, blocks, threads, iters, sink, stream=None):
    """Launch the FMA throughput microbenchmark (FP64 or, with precision MIXED, FP32) on the stream; returns
    the floating-point operations of the launch.  sink: CUDA tensor of blocks*threads elements of the type."""
    flops = C.c_double(0.0)
    _check(load().cloak_fma_peak(precision, blocks, threads, iters, C.c_void_p(sink.data_ptr()), C.byref(flops),
                                 _stream_ptr(stream)))
    return flops.value


def cloak_render_batch(h, views, spp, seed, stream=None):
    """views: list of (variant, polarization, eye, target, up, hfov_deg, out) with out a float32 CUDA tensor
    of shape (height, width, 4).  Renders all of them in one pass (one persistent integration kernel)."""
    arr = (View * len(views))()
    for a, (variant, pol, eye, target, up, hfov, out) in zip(arr, views):
        a.variant, a.polarization = variant, pol
        a.eye[:], a.target[:], a.up[:] = list(map(float, eye)), list(map(float, target)), list(map(float, up))
        a.hfov_deg = hfov
        a.height, a.width = int(out.shape[0]), int(out.shape[1])
        a.dev_rgba = out.data_ptr()
    return _check(load().cloak_render_batch(h, C.cast(arr, C.c_void_p), len(views), spp, seed, _stream_ptr(stream)))


def cloak_render_noalloc(h, polarization, spp, seed, rgba, stream=None):
    """Allocation-free render (fixed library-owned device array; at most 1048576 samples per call)."""
    return _check(load().cloak_render_noalloc(h, polarization, spp, seed, C.c_void_p(rgba.data_ptr()),
                                              rgba.numel() * rgba.element_size(), _stream_ptr(stream)))


# ------------------------------------------------------------------ panels of the paper's figures
PANEL_ROOM, PANEL_METAL, PANEL_UNPOLARIZED, PANEL_POLARIZER_RIGHT, PANEL_POLARIZER_UP, PANEL_TOF = 0, 1, 2, 3, 4, 5
ANALYZER_NONE, ANALYZER_RIGHT, ANALYZER_UP = 0, 1, 2
FORM_FERMAT, FORM_HAMILTONIAN = 0, 1


def cloak_set_formulation(h, formulation):
    return _check(load().cloak_set_formulation(h, formulation))


def cloak_set_analyzer(h, analyzer):
    return _check(load().cloak_set_analyzer(h, analyzer))


def cloak_set_reflections(h, on):
    return _check(load().cloak_set_reflections(h, on))


def cloak_render_panel(h, panel, spp, seed, rgba, stream=None):
    return _check(load().cloak_render_panel(h, panel, spp, seed, C.c_void_p(rgba.data_ptr()),
                                            rgba.numel() * rgba.element_size(), _stream_ptr(stream)))


# ------------------------------------------------------------------ learned surrogate
SUR_NPARAMS = 200709
SUR_INFO_KEYS = ("loss_stage1", "loss_stage2", "lateral_fraction", "rays", "seconds", "seconds_tracing",
                 "optimizer_steps", "batch")


def cloak_surrogate_train(h, n_rays, seed=0, epochs=20, stream=None):
    return _check(load().cloak_surrogate_train(h, n_rays, seed, epochs, _stream_ptr(stream)))


def cloak_surrogate_save(h, path):
    return _check(load().cloak_surrogate_save(h, os.fsencode(path)))


def cloak_surrogate_load(h, path):
    return _check(load().cloak_surrogate_load(h, os.fsencode(path)))


def cloak_surrogate_set_gate(h, max_log10_err):
    return _check(load().cloak_surrogate_set_gate(h, max_log10_err))


def cloak_surrogate_info(h) -> dict:
    buf = (C.c_double * 8)()
    _check(load().cloak_surrogate_info(h, buf))
    return dict(zip(SUR_INFO_KEYS, list(buf)))


def cloak_surrogate_set_precision(h, fp16):
    """Inference operands of the handle's surrogate: False = BF16 (default), True = FP16."""
    return _check(load().cloak_surrogate_set_precision(h, 1 if fp16 else 0))


def cloak_surrogate_train_timing(h) -> dict:
    """Device timing of the last training: ms per stage-1 and stage-2 step, flops of a stage-1 step, batch."""
    buf = (C.c_double * 4)()
    _check(load().cloak_surrogate_train_timing(h, buf))
    return dict(zip(("ms_per_step_stage1", "ms_per_step_stage2", "flops_per_step_stage1", "batch"), list(buf)))


def cloak_surrogate_params(h, values=None) -> np.ndarray:
    """Get (values None) or set the flat FP32 parameter vector (per layer W_l then b_l)."""
    if values is None:
        out = np.zeros(SUR_NPARAMS, np.float32)
        _check(load().cloak_surrogate_params(h, out.ctypes.data_as(C.POINTER(C.c_float)), SUR_NPARAMS, 0))
        return out
    v = np.ascontiguousarray(values, dtype=np.float32)
    _check(load().cloak_surrogate_params(h, v.ctypes.data_as(C.POINTER(C.c_float)), v.size, 1))
    return v


def cloak_surrogate_forward(h, x, y, stream=None):
    """x: float32 CUDA tensor (n, 7); y: float32 CUDA tensor (n, 5)."""
    return _check(load().cloak_surrogate_forward(h, C.c_void_p(x.data_ptr()), x.shape[0], C.c_void_p(y.data_ptr()),
                                                 _stream_ptr(stream)))


def cloak_surrogate_step(h, x, t, stage=1, lr=0.0, grad=True, stream=None):
    """One batch (x (n, 7), t (n, 8) float32 CUDA tensors, n % 128 == 0): the gradient of the mean loss
    (flat numpy vector) and, with lr > 0, one Adam step."""
    g = np.zeros(SUR_NPARAMS, np.float32) if grad else None
    _check(load().cloak_surrogate_step(h, C.c_void_p(x.data_ptr()), C.c_void_p(t.data_ptr()), x.shape[0], stage, lr,
                                       g.ctypes.data_as(C.POINTER(C.c_float)) if grad else None,
                                       _stream_ptr(stream)))
    return g


# ------------------------------------------------------------------ convenience
def records_to_numpy(buf) -> np.ndarray:
    """Copy a device record buffer to a structured numpy array (cloak_record layout)."""
    return buf.cpu().numpy().view(np.uint8).view(RECORD_DTYPE)


class Cloak:
    """Owning wrapper around a cloak_t handle."""

    def __init__(self, variant=RADIAL, R1=0.5, R2=1.0, height=2.0):
        self.h = cloak_create(variant, R1, R2, height)
        self.width, self.height = 128, 96

    def close(self):
        if self.h is not None:
            cloak_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def camera(self, eye, target=(0, 0, 0), up=(0, 0, 1), hfov_deg=60.0, width=128, height=96):
        cloak_camera_set(self.h, eye, target, up, hfov_deg, width, height)
        self.width, self.height = width, height
        return self

    def integrator(self, kind=RK4, h_or_tol=1e-3, precision=FP64, max_steps=1_000_000):
        cloak_set_integrator(self.h, kind, h_or_tol, precision, max_steps)
        return self

    def schedule(self, schedule=SCHED_PLAIN, packet=0, steps_per_round=0):
        cloak_set_schedule(self.h, schedule, packet, steps_per_round)
        return self

    def stage_timing(self, on=True):
        cloak_set_stage_timing(self.h, on)
        return self

    def stage_times(self):
        return cloak_stage_times(self.h)

    def test_medium(self, eps_o, eps_e, c_hat):
        cloak_set_test_medium(self.h, eps_o, eps_e, c_hat)
        return self

    def scene_seed(self, seed):
        cloak_set_scene_seed(self.h, seed)
        return self

    def render(self, polarization, spp=1, seed=0, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.height, self.width, 4), dtype=torch.float32, device="cuda")
        cloak_render(self.h, polarization, spp, seed, out, stream)
        return out

    def formulation(self, formulation=FORM_FERMAT):
        """Ray equations: FORM_FERMAT (Eq. 2 / Eq. 8) or FORM_HAMILTONIAN (state (x, k))."""
        cloak_set_formulation(self.h, formulation)
        return self

    def analyzer(self, analyzer=ANALYZER_NONE):
        """Linear polariser in front of the camera (ANALYZER_NONE / _RIGHT / _UP)."""
        cloak_set_analyzer(self.h, analyzer)
        return self

    def reflections(self, on=True):
        """First-order reflections in the unpolarised and polariser panels."""
        cloak_set_reflections(self.h, 1 if on else 0)
        return self

    def panel(self, panel, spp=1, seed=0, out=None, stream=None):
        """One panel of the paper's figures (PANEL_*; PANEL_TOF: time-of-flight difference image)."""
        import torch
        if out is None:
            out = torch.empty((self.height, self.width, 4), dtype=torch.float32, device="cuda")
        cloak_render_panel(self.h, panel, spp, seed, out, stream)
        return out

    def render_records(self, polarization, spp=1, seed=0, out=None, stream=None):
        import torch
        n = self.width * self.height * spp
        if out is None:
            out = torch.empty(n * RECORD_BYTES, dtype=torch.uint8, device="cuda")
        cloak_render_records(self.h, polarization, spp, seed, out, stream)
        return out

    def eval_rhs(self, polarization, y, stream=None):
        """Derivative of each state (rows of y, shape (n, 6)) under the handle's ray equations."""
        import torch
        y = y.to(device="cuda", dtype=torch.float64).contiguous()
        dy = torch.empty_like(y)
        cloak_eval_rhs(self.h, polarization, y, y.shape[0], dy, stream)
        return dy

    def trace_rays(self, polarization, rays, out=None, stream=None):
        import torch
        rays = rays.to(device="cuda", dtype=torch.float64).contiguous()
        n = rays.shape[0]
        if out is None:
            out = torch.empty(max(n, 1) * RECORD_BYTES, dtype=torch.uint8, device="cuda")
        cloak_trace_rays(self.h, polarization, rays, n, out, stream)
        return out
