"""CPU FP64 oracle for the uniaxial-cloak ray tracer -- TEST INFRASTRUCTURE ONLY.

A ctypes front end over ``libcloak_oracle.so`` (plain C, FP64; source in
``cloak_oracle.c``).  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package.  The renderer never routes through it.

Each wrapper names the passage of Halimeh & Wegener (arXiv:1209.6038) it
follows; the C source carries the detail.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RADIAL, AZIMUTHAL, TEST_CONST = 0, 1, 100
FERMAT, HAMILTONIAN = 0, 1
ORDINARY, EXTRAORDINARY = 0, 1
RK4, DP45 = 0, 1
STATUS = {0: "MISSED", 1: "EXITED", 2: "HIT_METAL_EXITED", 3: "NO_TRANSMISSION", 4: "TIR",
          5: "STEP_LIMIT", 6: "SINGULAR", 7: "METAL_CAP"}
MISSED, EXITED, HIT_METAL_EXITED, NO_TRANSMISSION, TIR, STEP_LIMIT, SINGULAR, METAL_CAP = range(8)

RECORD_DTYPE = np.dtype([("exit_pos", "<f8", 3), ("exit_dir", "<f8", 3), ("tof", "<f8"), ("weight", "<f8"),
                         ("tile_id", "<i4"), ("status", "<i4"), ("steps", "<i4"), ("mode", "<i4")])
assert RECORD_DTYPE.itemsize == 80


class _Cloak(C.Structure):
    _fields_ = [("variant", C.c_int), ("R1", C.c_double), ("R2", C.c_double), ("H", C.c_double),
                ("eps_o_test", C.c_double), ("eps_e_test", C.c_double), ("c_test", C.c_double * 3),
                ("scene_seed", C.c_uint64), ("analyzer", C.c_double * 3), ("form", C.c_int)]


class _Integ(C.Structure):
    _fields_ = [("kind", C.c_int), ("h_or_tol", C.c_double), ("max_steps", C.c_long)]


class _Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("target", C.c_double * 3), ("up", C.c_double * 3),
                ("hfov_deg", C.c_double), ("width", C.c_int), ("height", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_splitmix64.argtypes = [C.c_uint64]
        L.orc_uniform.restype = C.c_double
        L.orc_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32]
        L.orc_permittivity.argtypes = [C.POINTER(_Cloak), dp, dp, dp, dp, dp]
        L.orc_aux_matrix.argtypes = [C.POINTER(_Cloak), dp, dp, dp]
        L.orc_aux_inverse.argtypes = [C.POINTER(_Cloak), dp, dp]
        L.orc_eq8_accel.argtypes = [dp, dp, dp, dp]
        L.orc_eq2_accel.argtypes = [C.c_double, dp, dp, dp]
        L.orc_rhs.argtypes = [C.POINTER(_Cloak), C.c_int, dp, dp]
        L.orc_refract_into.restype = C.c_int
        L.orc_refract_into.argtypes = [C.POINTER(_Cloak), C.c_int, dp, dp, dp, dp, dp]
        L.orc_mode_fields.argtypes = [C.POINTER(_Cloak), C.c_int, dp, dp, dp, dp, dp]
        L.orc_transmission_in.restype = C.c_int
        L.orc_transmission_in.argtypes = [C.POINTER(_Cloak), dp, dp, dp, dp]
        L.orc_transmission_out.restype = C.c_int
        L.orc_transmission_out.argtypes = [C.POINTER(_Cloak), C.c_int, dp, dp, dp, dp]
        L.orc_rk4_step.argtypes = [C.POINTER(_Cloak), C.c_int, dp, C.c_double, dp]
        L.orc_dp45_step.argtypes = [C.POINTER(_Cloak), C.c_int, dp, C.c_double, dp, dp]
        L.orc_trace_ray.restype = C.c_int
        L.orc_trace_ray.argtypes = [C.POINTER(_Cloak), C.POINTER(_Integ), C.c_int, dp, dp, C.c_void_p,
                                    dp, C.c_long, C.POINTER(C.c_long)]
        L.orc_trace_rays.argtypes = [C.POINTER(_Cloak), C.POINTER(_Integ), C.c_int, dp, C.c_long, C.c_void_p,
                                     C.c_int]
        L.orc_camera_ray.argtypes = [C.POINTER(_Camera), C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, dp, dp]
        L.orc_shade.restype = C.c_int
        L.orc_shade.argtypes = [C.POINTER(_Cloak), dp, dp, dp]
        L.orc_render.argtypes = [C.POINTER(_Cloak), C.POINTER(_Integ), C.POINTER(_Camera), C.c_int, C.c_int,
                                 C.c_uint64, C.POINTER(C.c_int64), C.c_long, dp, C.c_void_p, C.c_int]
        L.orc_rhs_hamiltonian.argtypes = [C.POINTER(_Cloak), C.c_int, dp, dp]
        L.orc_trace_reflections.restype = C.c_int
        L.orc_trace_reflections.argtypes = [C.POINTER(_Cloak), C.POINTER(_Integ), C.c_int, dp, dp, C.c_void_p,
                                            C.c_void_p]
        L.orc_room_distance.restype = C.c_double
        L.orc_room_distance.argtypes = [C.POINTER(_Cloak), dp, dp]
        L.orc_tof_difference.restype = C.c_double
        L.orc_tof_difference.argtypes = [C.POINTER(_Cloak), dp, dp, C.c_void_p]
        # surrogate (surrogate_oracle.h)
        ip = C.POINTER(C.c_int)
        L.orc_gelu.restype = C.c_double
        L.orc_gelu.argtypes = [C.c_double]
        L.orc_gelu_grad.restype = C.c_double
        L.orc_gelu_grad.argtypes = [C.c_double]
        L.orc_mlp_nparams.restype = C.c_long
        L.orc_mlp_nparams.argtypes = [C.c_int, ip]
        L.orc_mlp_forward.argtypes = [C.c_int, ip, dp, C.c_long, dp, dp]
        L.orc_mlp_backward.argtypes = [C.c_int, ip, dp, C.c_long, dp, dp, dp]
        L.orc_sur_loss.restype = C.c_double
        L.orc_sur_loss.argtypes = [C.c_int, C.c_long, dp, dp, dp, dp]
        L.orc_adam_step.argtypes = [C.c_long, dp, dp, dp, dp, C.c_long, C.c_double, C.c_double, C.c_double,
                                    C.c_double]
        L.orc_sur_sample.argtypes = [C.c_uint64, C.c_uint64, C.c_double, C.c_double, dp, dp, ip, ip]
        L.orc_sur_features.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, dp, dp, dp]
        L.orc_sur_targets.restype = C.c_int
        L.orc_sur_targets.argtypes = [C.c_double, C.c_double, dp, dp, C.c_void_p, dp]
        L.orc_sur_reconstruct.argtypes = [C.c_double, C.c_double, dp, dp, dp, dp, dp, dp]
        _lib = L
    return _lib


_ext_libs = {}


def ext_lib(kind: str = "ld"):
    """The same oracle source built in extended precision (kind "ld": long double, "q": _Float128), for the
    rays FP64 cannot determine.  Only orc_render and orc_trace_rays are bound: their arguments are FP64 in
    every build (inputs exact, outputs rounded once at the end)."""
    if kind not in _ext_libs:
        L = C.CDLL(_build.build_ext(kind))
        L.orc_trace_rays.argtypes = [C.POINTER(_Cloak), C.POINTER(_Integ), C.c_int, C.POINTER(C.c_double),
                                     C.c_long, C.c_void_p, C.c_int]
        L.orc_render.argtypes = [C.POINTER(_Cloak), C.POINTER(_Integ), C.POINTER(_Camera), C.c_int, C.c_int,
                                 C.c_uint64, C.POINTER(C.c_int64), C.c_long, C.POINTER(C.c_double), C.c_void_p,
                                 C.c_int]
        _ext_libs[kind] = L
    return _ext_libs[kind]


def _select(precision):
    return lib() if precision == "f64" else ext_lib(precision)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(x, n=3):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))
    return a


class Cloak:
    """Cloak geometry and material: Eq. 14 (radial) or Eq. 15 (azimuthal), or a
    homogeneous uniaxial test medium (Eq. 1 with a fixed optic axis)."""

    def __init__(self, variant=RADIAL, R1=0.5, R2=1.0, H=2.0, eps_o=1.0, eps_e=1.0, c_hat=(0, 0, 1),
                 scene_seed=0, analyzer=(0.0, 0.0, 0.0), form=0):
        """analyzer: axis of a linear polariser in front of the camera (zero: none); form: ray equations
        (0 Fermat form, Eq. 2 / Eq. 8; 1 Hamiltonian form)."""
        self.s = _Cloak(variant, R1, R2, H, eps_o, eps_e, (C.c_double * 3)(*c_hat), scene_seed,
                        (C.c_double * 3)(*analyzer), form)

    @property
    def ref(self):
        return C.byref(self.s)


class Integrator:
    """RK4 at fixed step h (Sect. 4) or Dormand-Prince 5(4) at tolerance tol."""

    def __init__(self, kind=RK4, h_or_tol=1e-3, max_steps=2_000_000):
        self.s = _Integ(kind, h_or_tol, max_steps)

    @property
    def ref(self):
        return C.byref(self.s)


class Camera:
    def __init__(self, eye, target=(0, 0, 0), up=(0, 0, 1), hfov_deg=60.0, width=128, height=96):
        self.s = _Camera((C.c_double * 3)(*eye), (C.c_double * 3)(*target), (C.c_double * 3)(*up), hfov_deg,
                         width, height)
        self.width, self.height = width, height

    @property
    def ref(self):
        return C.byref(self.s)


def splitmix64(z: int) -> int:
    return int(lib().orc_splitmix64(z & 0xFFFFFFFFFFFFFFFF))


def uniform(seed, pixel, sample, dim) -> float:
    return float(lib().orc_uniform(seed, pixel, sample, dim))


def permittivity(cloak: Cloak, x):
    x = _vec(x)
    eps = np.zeros(9)
    eo, ee = C.c_double(), C.c_double()
    ch = np.zeros(3)
    lib().orc_permittivity(cloak.ref, _dp(x), _dp(eps), C.byref(eo), C.byref(ee), _dp(ch))
    return eps.reshape(3, 3), eo.value, ee.value, ch


def aux_matrix(cloak: Cloak, x):
    """Eq. 7: M and dM[k, i, j] = d M_ij / d x_k."""
    x = _vec(x)
    M = np.zeros(9)
    dM = np.zeros(27)
    lib().orc_aux_matrix(cloak.ref, _dp(x), _dp(M), _dp(dM))
    return M.reshape(3, 3), dM.reshape(3, 3, 3)


def aux_inverse(cloak: Cloak, x):
    """Eq. 7 inverted: M^{-1} = eps / (n_o^2 n_e^2)."""
    x = _vec(x)
    Mi = np.zeros(9)
    lib().orc_aux_inverse(cloak.ref, _dp(x), _dp(Mi))
    return Mi.reshape(3, 3)


def eq8_accel(Minv, dM, v):
    """Eq. 8 given M^{-1} and the gradient of M."""
    M = np.ascontiguousarray(Minv, dtype=np.float64).reshape(9)
    dM = np.ascontiguousarray(dM, dtype=np.float64).reshape(27)
    v = _vec(v)
    a = np.zeros(3)
    lib().orc_eq8_accel(_dp(M), _dp(dM), _dp(v), _dp(a))
    return a


def eq2_accel(n, gradn, v):
    g = _vec(gradn)
    v = _vec(v)
    a = np.zeros(3)
    lib().orc_eq2_accel(float(n), _dp(g), _dp(v), _dp(a))
    return a


def rhs(cloak: Cloak, mode, y):
    y = _vec(y, 6)
    dy = np.zeros(6)
    lib().orc_rhs(cloak.ref, mode, _dp(y), _dp(dy))
    return dy


def rhs_hamiltonian(cloak: Cloak, mode, y):
    """d(x, k)/dt of the Hamiltonian form (state y = (x, k), k = M v)."""
    y = _vec(y, 6)
    dy = np.zeros(6)
    lib().orc_rhs_hamiltonian(cloak.ref, mode, _dp(y), _dp(dy))
    return dy


def refract_into(cloak: Cloak, mode, x, n, kt):
    """Sect. 3, Eqs. 9-11: inward wave of the mode with tangential wave vector kt.
    Returns (k, v) or None when the mode is evanescent."""
    x, n, kt = _vec(x), _vec(n), _vec(kt)
    k = np.zeros(3)
    v = np.zeros(3)
    ok = lib().orc_refract_into(cloak.ref, mode, _dp(x), _dp(n), _dp(kt), _dp(k), _dp(v))
    return (k, v) if ok else None


def mode_fields(cloak: Cloak, mode, x, k):
    """Sect. 3 field directions (D, E, H) of the propagating wave with wave vector k."""
    x, k = _vec(x), _vec(k)
    D, E, H = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_mode_fields(cloak.ref, mode, _dp(x), _dp(k), _dp(D), _dp(E), _dp(H))
    return D, E, H


def transmission_in(cloak: Cloak, x, n, d):
    """Eq. 12 vacuum -> medium: dict of T_o^s, T_o^p, T_e^s, T_e^p, R^s, R^p, T_o, T_e."""
    x, n, d = _vec(x), _vec(n), _vec(d)
    out = np.zeros(8)
    ok = lib().orc_transmission_in(cloak.ref, _dp(x), _dp(n), _dp(d), _dp(out))
    keys = ["To_s", "To_p", "Te_s", "Te_p", "R_s", "R_p", "To", "Te"]
    return dict(zip(keys, out)) if ok else None


def transmission_out(cloak: Cloak, mode, x, n, k):
    """Eq. 12 medium -> vacuum: (ok, T, R_o, R_e); under total internal reflection T = 0, R_o + R_e = 1."""
    x, n, k = _vec(x), _vec(n), _vec(k)
    out = np.zeros(4)
    ok = lib().orc_transmission_out(cloak.ref, mode, _dp(x), _dp(n), _dp(k), _dp(out))
    return bool(ok), out[0], out[1], out[2]


def analyzer_fraction(cloak: Cloak, mode, x, n, k):
    """Fraction of the flux transmitted into vacuum that passes the cloak's analyser (cloak.s.analyzer)."""
    x, n, k = _vec(x), _vec(n), _vec(k)
    out = np.zeros(4)
    ok = lib().orc_transmission_out(cloak.ref, mode, _dp(x), _dp(n), _dp(k), _dp(out))
    return out[3] if ok else None


def rk4_step(cloak: Cloak, mode, y, h):
    y = _vec(y, 6)
    o = np.zeros(6)
    lib().orc_rk4_step(cloak.ref, mode, _dp(y), float(h), _dp(o))
    return o


def dp45_step(cloak: Cloak, mode, y, h):
    y = _vec(y, 6)
    o = np.zeros(6)
    e = np.zeros(6)
    lib().orc_dp45_step(cloak.ref, mode, _dp(y), float(h), _dp(o), _dp(e))
    return o, e


def trace_ray(cloak: Cloak, integ: Integrator, mode, o, d, path_cap=0):
    """One ray through entry split, integration, exit refraction and shading.
    Returns (record, path) where path rows are (t, x, y, z, vx, vy, vz)."""
    o, d = _vec(o), _vec(d)
    rec = np.zeros(1, dtype=RECORD_DTYPE)
    path = np.zeros((max(path_cap, 1), 7))
    plen = C.c_long(0)
    lib().orc_trace_ray(cloak.ref, integ.ref, mode, _dp(o), _dp(d), rec.ctypes.data_as(C.c_void_p),
                        _dp(path) if path_cap > 0 else None, path_cap, C.byref(plen))
    return rec[0], path[: min(plen.value, path_cap)]


def trace_rays(cloak: Cloak, integ: Integrator, mode, rays, nthreads=None, precision="f64"):
    """precision: "f64" (the oracle), or "ld" / "q" (the same source in extended precision)."""
    rays = np.ascontiguousarray(rays, dtype=np.float64).reshape(-1, 6)
    n = rays.shape[0]
    recs = np.zeros(n, dtype=RECORD_DTYPE)
    _select(precision).orc_trace_rays(cloak.ref, integ.ref, mode, _dp(rays), n, recs.ctypes.data_as(C.c_void_p),
                         nthreads or os.cpu_count() or 1)
    return recs


def camera_ray(cam: Camera, i, j, s, spp, seed):
    o = np.zeros(3)
    d = np.zeros(3)
    lib().orc_camera_ray(cam.ref, i, j, s, spp, seed, _dp(o), _dp(d))
    return o, d


def shade(cloak: Cloak, p, d):
    p, d = _vec(p), _vec(d)
    rgb = np.zeros(3)
    tile = lib().orc_shade(cloak.ref, _dp(p), _dp(d), _dp(rgb))
    return tile, rgb


def render(cloak: Cloak, integ: Integrator, cam: Camera, mode, spp=1, seed=0, pixels=None, nthreads=None,
           records=True, precision="f64"):
    """Whole image (or a pixel subset, flat indices j*W+i): RGBA = mean over samples of
    weight * colour (alpha = mean weight) and per-sample records.  precision: "f64" (the oracle), or
    "ld" / "q" (the same source in extended precision)."""
    if pixels is None:
        npix = cam.width * cam.height
        pix_ptr = None
    else:
        pixels = np.ascontiguousarray(pixels, dtype=np.int64)
        npix = pixels.shape[0]
        pix_ptr = pixels.ctypes.data_as(C.POINTER(C.c_int64))
    rgba = np.zeros((npix, 4))
    recs = np.zeros(npix * spp, dtype=RECORD_DTYPE) if records else None
    _select(precision).orc_render(cloak.ref, integ.ref, cam.ref, mode, spp, seed, pix_ptr, npix, _dp(rgba),
                     recs.ctypes.data_as(C.c_void_p) if records else None, nthreads or os.cpu_count() or 1)
    return rgba, recs


def trace_reflections(cloak: Cloak, integ: Integrator, mode, o, d):
    """First-order reflections of a camera sample traced in `mode`: (vac, refl) records, vac the room light
    the outer surface reflects into the camera, refl[m'] the light that travelled as mode m' and reflected
    at the far face into `mode`."""
    vac = np.zeros(1, dtype=RECORD_DTYPE)
    refl = np.zeros(2, dtype=RECORD_DTYPE)
    lib().orc_trace_reflections(cloak.ref, integ.ref, mode, _dp(_vec(o)), _dp(_vec(d)),
                                vac.ctypes.data_as(C.c_void_p), refl.ctypes.data_as(C.c_void_p))
    return vac[0], refl


def reflections_image(cloak: Cloak, integ: Integrator, cam: Camera, spp=1, seed=0, pixels=None):
    """Per pixel, the first-order reflections' part of the unpolarised panel (Fig. 1 (c) / 2 (c)): the mean
    over samples of the outer-surface reflection (once) plus the far-face reflections of both traced modes
    (each into o and e), weight x room colour; RGB and summed weight."""
    idx = np.arange(cam.width * cam.height) if pixels is None else np.asarray(pixels)
    out = np.zeros((len(idx), 4))
    for n, pix in enumerate(idx):
        i, j = int(pix) % cam.width, int(pix) // cam.width
        acc = np.zeros(4)
        for s in range(spp):
            o, d = camera_ray(cam, i, j, s, spp, seed)
            recs = []
            for mode in (ORDINARY, EXTRAORDINARY):
                vac, refl = trace_reflections(cloak, integ, mode, o, d)
                recs += list(refl)
            recs.append(vac)
            for r in recs:
                if r["weight"] > 0.0:
                    _, rgb = shade(cloak, r["exit_pos"], r["exit_dir"])
                    acc[:3] += r["weight"] * np.asarray(rgb)
                    acc[3] += r["weight"]
        out[n] = acc / spp
    return out


def camera_axes(cam: Camera):
    """The pinhole camera's right and up unit vectors (the frame orc_camera_ray builds: w towards the target,
    right = w x up normalised, up' = right x w)."""
    e = np.array(cam.s.eye[:])
    w = np.array(cam.s.target[:]) - e
    w /= np.linalg.norm(w)
    u = np.cross(w, np.array(cam.s.up[:]))
    u /= np.linalg.norm(u)
    return u, np.cross(u, w)


PANELS = ("unpolarized", "polarizer_right", "polarizer_up")


def panel_image(variant, integ: Integrator, cam: Camera, kind="unpolarized", spp=1, seed=0, pixels=None,
                reflections=False, R1=0.5, R2=1.0, H=2.0, nthreads=None):
    """Panels (c)-(e) of Figs. 1 and 2 (Sect. 4; Sect. 5 for the polariser): the cloak seen in unpolarised room
    light ("unpolarized"), or through a linear polariser in front of the camera whose axis is the camera's
    right ("polarizer_right") or up ("polarizer_up") vector.  Per sample, the light arriving as the ordinary
    and as the extraordinary wave add incoherently, each with its own Eq. 12 factors (and the polariser's
    Malus factor); a sample that never enters the shell -- it misses the cylinder or mirrors off a metal end
    disc -- is the same room light for both and counts once.  reflections: add the first-order reflections
    (the outer surface's, once, and the far-face reflections of both waves: reflections_image).
    Per pixel: RGB = mean over samples of weight x room colour, A = mean summed weight."""
    if kind not in PANELS:
        raise ValueError(kind)
    axis = (0.0, 0.0, 0.0)
    if kind != "unpolarized":
        right, up = camera_axes(cam)
        axis = tuple(right if kind == "polarizer_right" else up)
    cl = Cloak(variant, R1=R1, R2=R2, H=H, analyzer=axis)
    _, ro = render(cl, integ, cam, ORDINARY, spp, seed, pixels, nthreads)
    _, re = render(cl, integ, cam, EXTRAORDINARY, spp, seed, pixels, nthreads)
    n = len(ro) // spp
    out = np.zeros((n, 4))
    for k in range(n * spp):
        a, b = ro[k], re[k]
        enters = a["status"] not in (MISSED, METAL_CAP)
        for r in ((a, b) if enters else (a,)):
            if r["weight"] > 0.0 and r["tile_id"] >= 0:
                _, rgb = shade(cl, r["exit_pos"], r["exit_dir"])
                out[k // spp, :3] += r["weight"] * np.asarray(rgb)
            out[k // spp, 3] += r["weight"]
    out /= spp
    if reflections:
        out += reflections_image(cl, integ, cam, spp, seed, pixels)
    return out


def room_distance(cloak: Cloak, p, d) -> float:
    return lib().orc_room_distance(cloak.ref, _dp(_vec(p)), _dp(_vec(d)))


def tof_difference(cloak: Cloak, o, d, rec) -> float:
    """Time of flight of the light one camera sample receives minus the time without the cylinder."""
    r = np.array(rec, dtype=RECORD_DTYPE).reshape(1)
    return lib().orc_tof_difference(cloak.ref, _dp(_vec(o)), _dp(_vec(d)), r.ctypes.data_as(C.c_void_p))


def tof_image(cloak: Cloak, integ: Integrator, cam: Camera, spp=1, seed=0, pixels=None, nthreads=None):
    """Time-of-flight difference image (Sect. 4; the TOF images of Ref. [10]), per pixel:
    (0) intensity-weighted mean TOF difference of the light of both polarizations, (1) of the ordinary
    and (2) of the extraordinary light alone, (3) the summed weight (mean over samples).  A sample that
    never enters the shell (it misses the cylinder or mirrors off a metal end disc) is the same light in
    both polarizations and counts once in (0) and (3).  The weights include the camera polariser
    (cloak analyzer) when one is set; a pixel without light gets 0."""
    _, ro = render(cloak, integ, cam, ORDINARY, spp, seed, pixels, nthreads)
    _, re = render(cloak, integ, cam, EXTRAORDINARY, spp, seed, pixels, nthreads)
    idx = np.arange(cam.width * cam.height) if pixels is None else np.asarray(pixels)
    out = np.zeros((len(idx), 4))
    for n, pix in enumerate(idx):
        i, j = int(pix) % cam.width, int(pix) // cam.width
        A = W = Ao = Wo = Ae = We = 0.0
        for s in range(spp):
            o, d = camera_ray(cam, i, j, s, spp, seed)
            a, b = ro[n * spp + s], re[n * spp + s]
            dto, dte = tof_difference(cloak, o, d, a), tof_difference(cloak, o, d, b)
            enters = a["status"] not in (MISSED, METAL_CAP)
            Ao += a["weight"] * dto
            Wo += a["weight"]
            Ae += b["weight"] * dte
            We += b["weight"]
            A += a["weight"] * dto + (b["weight"] * dte if enters else 0.0)
            W += a["weight"] + (b["weight"] if enters else 0.0)
        out[n] = (A / W if W > 0 else 0.0, Ao / Wo if Wo > 0 else 0.0, Ae / We if We > 0 else 0.0, W / spp)
    return out


# ------------------------------------------------------------------ learned surrogate (surrogate_oracle.h)
SUR_DIMS = (7, 256, 256, 256, 256, 5)


def _dims(dims):
    d = np.ascontiguousarray(dims, dtype=np.int32)
    return len(dims) - 1, d, d.ctypes.data_as(C.POINTER(C.c_int))


def gelu(x: float) -> float:
    return lib().orc_gelu(float(x))


def gelu_grad(x: float) -> float:
    return lib().orc_gelu_grad(float(x))


def mlp_nparams(dims) -> int:
    nl, d, dptr = _dims(dims)
    return lib().orc_mlp_nparams(nl, dptr)


def mlp_split(dims, params):
    """[(W_l, b_l)] views of a flat parameter vector (W_l: dims[l+1] x dims[l])."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        nw = dims[l + 1] * dims[l]
        out.append((params[o:o + nw].reshape(dims[l + 1], dims[l]), params[o + nw:o + nw + dims[l + 1]]))
        o += nw + dims[l + 1]
    return out


def mlp_forward(dims, params, x):
    nl, d, dptr = _dims(dims)
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, dims[0])
    y = np.zeros((x.shape[0], dims[-1]))
    lib().orc_mlp_forward(nl, dptr, _dp(params), x.shape[0], _dp(x), _dp(y))
    return y


def mlp_backward(dims, params, x, dy):
    """Gradient of sum(dy * network(x)) with respect to the flat parameters."""
    nl, d, dptr = _dims(dims)
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, dims[0])
    dy = np.ascontiguousarray(dy, dtype=np.float64).reshape(-1, dims[-1])
    g = np.zeros_like(params)
    lib().orc_mlp_backward(nl, dptr, _dp(params), x.shape[0], _dp(x), _dp(dy), _dp(g))
    return g


def sur_loss(stage, y, t, mask):
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(-1, 5)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1, 5)
    mask = np.ascontiguousarray(mask, dtype=np.float64).reshape(-1)
    dy = np.zeros_like(y)
    L = lib().orc_sur_loss(stage, y.shape[0], _dp(y), _dp(t), _dp(mask), _dp(dy))
    return L, dy


def adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on p, m, v (float64 contiguous arrays)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam_step(p.size, _dp(p), _dp(g), _dp(m), _dp(v), step, lr, beta1, beta2, eps)


def sur_sample(seed, i, R2=1.0, H=2.0):
    P, d = np.zeros(3), np.zeros(3)
    mode, variant = C.c_int(0), C.c_int(0)
    lib().orc_sur_sample(seed, i, R2, H, _dp(P), _dp(d), C.byref(mode), C.byref(variant))
    return P, d, mode.value, variant.value


def sur_features(R1, R2, H, variant, mode, P, d):
    x = np.zeros(7)
    lib().orc_sur_features(R1, R2, H, variant, mode, _dp(_vec(P)), _dp(_vec(d)), _dp(x))
    return x


def sur_targets(R2, H, P, d, rec):
    """(lateral, t[4]) of a traced record (numpy RECORD_DTYPE scalar)."""
    r = np.array([rec], dtype=RECORD_DTYPE)
    t = np.zeros(4)
    ok = lib().orc_sur_targets(R2, H, _dp(_vec(P)), _dp(_vec(d)), r.ctypes.data_as(C.c_void_p), _dp(t))
    return bool(ok), t


def sur_reconstruct(R2, H, P, d, y):
    y = np.ascontiguousarray(y[:4], dtype=np.float64)
    pos, dr, tof = np.zeros(3), np.zeros(3), C.c_double(0)
    lib().orc_sur_reconstruct(R2, H, _dp(_vec(P)), _dp(_vec(d)), _dp(y), _dp(pos), _dp(dr), C.byref(tof))
    return pos, dr, tof.value
