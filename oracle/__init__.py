"""ctypes wrapper of the FP64 CPU oracle (``vr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()`` and by the
benchmark's CPU-baseline leg, never by the product package.  It shares no code with the
CUDA path.  See the header of ``vr_oracle.c`` for the method and the readings it follows.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py`` and
``tests/test_oracle_surface_pins.py`` except the Zucker-Hummel weights, whose agreement with
the paper's own operator is "parity unpinned" (the paper does not print that mask).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

GRAD = {"central": 0, "sobel3d": 1, "zucker_hummel": 2}
_DT = {np.dtype(np.uint8): 0, np.dtype(np.uint16): 1, np.dtype(np.float32): 2,
       np.dtype(np.float64): 3}


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("ortho", C.c_int), ("fov_y_deg", C.c_float), ("ortho_height", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class Params(C.Structure):
    _fields_ = [("step", C.c_float), ("grad", C.c_int), ("ka", C.c_double), ("kd", C.c_double),
                ("ks", C.c_double), ("shininess", C.c_double), ("light", C.c_double * 3),
                ("headlight", C.c_int), ("ert_threshold", C.c_double),
                ("clip_lo", C.c_float * 3), ("clip_hi", C.c_float * 3),
                ("adapt_range2", C.c_double), ("adapt_range4", C.c_double)]


class SurfaceParams(C.Structure):
    _fields_ = [("step", C.c_float), ("iso_lo", C.c_float), ("iso_hi", C.c_float),
                ("refine", C.c_int), ("grad", C.c_int), ("ka", C.c_double), ("kd", C.c_double),
                ("ks", C.c_double), ("shininess", C.c_double), ("light", C.c_double * 3),
                ("headlight", C.c_int), ("color", C.c_double * 3),
                ("clip_lo", C.c_float * 3), ("clip_hi", C.c_float * 3)]


class Volume(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int), ("n", C.c_int * 3),
                ("value_max", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.vro_sample.restype = C.c_double
        L.vro_sample.argtypes = [C.POINTER(Volume), dp]
        L.vro_gradient.argtypes = [C.POINTER(Volume), C.c_int, dp, dp]
        L.vro_tf.argtypes = [dp, C.c_int, C.c_double, dp, dp]
        L.vro_shade.argtypes = [dp, dp, dp, dp, C.c_double, C.c_double, C.c_double, C.c_double, dp]
        L.vro_composite.restype = C.c_int
        L.vro_composite.argtypes = [dp, dp, C.c_int, C.c_double, dp]
        L.vro_ray.restype = C.c_int
        L.vro_ray.argtypes = [C.POINTER(Camera), C.POINTER(Params), C.POINTER(C.c_int), C.c_int,
                              C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float),
                              C.POINTER(C.c_float), C.POINTER(C.c_int)]
        L.vro_render.restype = C.c_longlong
        L.vro_render.argtypes = [C.POINTER(Volume), dp, C.c_int, C.POINTER(Camera),
                                 C.POINTER(Params), dp, C.POINTER(C.c_int), C.c_int, C.c_int,
                                 C.c_int]
        L.vro_render_pixels.restype = C.c_longlong
        L.vro_render_pixels.argtypes = [C.POINTER(Volume), dp, C.c_int, C.POINTER(Camera),
                                        C.POINTER(Params), C.POINTER(C.c_int),
                                        C.POINTER(C.c_int), C.c_int, dp, C.POINTER(C.c_int),
                                        C.c_int]
        L.vro_num_threads.restype = C.c_int
        L.vro_sample_f32.restype = C.c_float
        L.vro_sample_f32.argtypes = [C.POINTER(Volume), C.POINTER(C.c_float)]
        L.vro_render_surface.restype = C.c_longlong
        L.vro_render_surface.argtypes = [C.POINTER(Volume), C.POINTER(Camera),
                                         C.POINTER(SurfaceParams), dp, C.POINTER(C.c_float),
                                         C.c_int, C.c_int, C.c_int]
        L.vro_render_backward.argtypes = [C.POINTER(Volume), dp, C.c_int, C.POINTER(Camera),
                                          C.POINTER(Params), dp, dp, dp]
        _lib = L
    return _lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleVolume:
    """Keeps the numpy buffer alive behind the C struct.  ``vol`` has shape (nz, ny, nx)."""

    def __init__(self, vol: np.ndarray, value_max: float):
        vol = np.asarray(vol)
        if vol.dtype == np.float16:
            vol = vol.astype(np.float32)  # exact widening
        if vol.dtype not in _DT:
            vol = vol.astype(np.float64)
        self.arr = np.ascontiguousarray(vol)
        nz, ny, nx = self.arr.shape
        self.s = Volume(self.arr.ctypes.data, _DT[self.arr.dtype], (C.c_int * 3)(nx, ny, nz),
                        float(value_max))
        self.shape_xyz = (nx, ny, nz)


def make_camera(cam: dict) -> Camera:
    return Camera((C.c_float * 3)(*cam["eye"]), (C.c_float * 3)(*cam["target"]),
                  (C.c_float * 3)(*cam["up"]), int(bool(cam["ortho"])), float(cam["fov_y_deg"]),
                  float(cam["ortho_height"]), int(cam["width"]), int(cam["height"]))


def make_params(step=0.5, grad="central", ka=0.1, kd=0.7, ks=0.2, shininess=20.0,
                light=(0.0, 0.0, 0.0), headlight=True, ert_threshold=0.99,
                clip_lo=(-1e30, -1e30, -1e30), clip_hi=(1e30, 1e30, 1e30),
                adapt_range=(-1.0, -1.0)) -> Params:
    """adapt_range = (range bound of multiplier 2, range bound of multiplier 4), raw units;
    negative = that level off (reading R16)."""
    g = GRAD[grad] if isinstance(grad, str) else int(grad)
    return Params(float(step), g, ka, kd, ks, shininess, (C.c_double * 3)(*light),
                  int(bool(headlight)), ert_threshold, (C.c_float * 3)(*clip_lo),
                  (C.c_float * 3)(*clip_hi), float(adapt_range[0]), float(adapt_range[1]))


def sample(ov: OracleVolume, p) -> float:
    p = np.ascontiguousarray(p, np.float64)
    return lib().vro_sample(C.byref(ov.s), _dptr(p))


def gradient(ov: OracleVolume, grad, p) -> np.ndarray:
    p = np.ascontiguousarray(p, np.float64)
    g = np.zeros(3)
    lib().vro_gradient(C.byref(ov.s), GRAD[grad] if isinstance(grad, str) else grad, _dptr(p),
                       _dptr(g))
    return g


def tf_lookup(tf, s):
    tf = np.ascontiguousarray(tf, np.float64)
    out, slope = np.zeros(4), np.zeros(4)
    lib().vro_tf(_dptr(tf), tf.shape[0], float(s), _dptr(out), _dptr(slope))
    return out, slope


def shade(N, L, V, rgb, ka=0.1, kd=0.7, ks=0.2, shininess=20.0):
    arrs = [np.ascontiguousarray(a, np.float64) for a in (N, L, V, rgb)]
    c = np.zeros(3)
    lib().vro_shade(*[_dptr(a) for a in arrs], ka, kd, ks, shininess, _dptr(c))
    return c


def composite(alpha, rgb, ert=0.99):
    alpha = np.ascontiguousarray(alpha, np.float64)
    rgb = np.ascontiguousarray(rgb, np.float64).reshape(-1, 3)
    out = np.zeros(4)
    n = lib().vro_composite(_dptr(alpha), _dptr(rgb), alpha.shape[0], ert, _dptr(out))
    return out, n


def ray(cam: dict, params: Params, shape_xyz, px, py):
    o = (C.c_float * 3)()
    d = (C.c_float * 3)()
    tn = C.c_float()
    K = C.c_int()
    n = (C.c_int * 3)(*shape_xyz)
    hit = lib().vro_ray(C.byref(make_camera(cam)), C.byref(params), n, px, py, o, d,
                        C.byref(tn), C.byref(K))
    return bool(hit), np.array(o[:], np.float32), np.array(d[:], np.float32), np.float32(tn.value), K.value


def render(ov: OracleVolume, tf, cam: dict, params: Params, rows=None, nthreads=0):
    """Render the image (or rows [r0, r1)).  Returns (rgba HxWx4 float64, counts HxW, total)."""
    tf = np.ascontiguousarray(tf, np.float64)
    H, W = cam["height"], cam["width"]
    r0, r1 = (0, H) if rows is None else rows
    out = np.zeros((H, W, 4))
    counts = np.zeros((H, W), np.int32)
    total = lib().vro_render(C.byref(ov.s), _dptr(tf), tf.shape[0], C.byref(make_camera(cam)),
                             C.byref(params), _dptr(out), counts.ctypes.data_as(C.POINTER(C.c_int)),
                             r0, r1, nthreads)
    return out, counts, int(total)


def render_pixels(ov: OracleVolume, tf, cam: dict, params: Params, px, py, nthreads=0):
    tf = np.ascontiguousarray(tf, np.float64)
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    out = np.zeros((px.shape[0], 4))
    counts = np.zeros(px.shape[0], np.int32)
    ip = C.POINTER(C.c_int)
    total = lib().vro_render_pixels(C.byref(ov.s), _dptr(tf), tf.shape[0],
                                    C.byref(make_camera(cam)), C.byref(params),
                                    px.ctypes.data_as(ip), py.ctypes.data_as(ip), px.shape[0],
                                    _dptr(out), counts.ctypes.data_as(ip), nthreads)
    return out, counts, int(total)


def render_backward(ov: OracleVolume, tf, cam: dict, params: Params, grad_rgba):
    """FP64 reverse mode.  Returns (dL/d raw voxels (nz,ny,nx), dL/dTF (n,4))."""
    tf = np.ascontiguousarray(tf, np.float64)
    g = np.ascontiguousarray(grad_rgba, np.float64)
    gv = np.zeros(ov.arr.shape)
    gt = np.zeros(tf.shape)
    lib().vro_render_backward(C.byref(ov.s), _dptr(tf), tf.shape[0], C.byref(make_camera(cam)),
                              C.byref(params), _dptr(g), _dptr(gv), _dptr(gt))
    return gv, gt


def num_threads() -> int:
    return lib().vro_num_threads()


def make_surface_params(step=2.0, iso_lo=0.5, iso_hi=1e30, refine=6, grad="central", ka=0.1,
                        kd=0.7, ks=0.2, shininess=20.0, light=(0.0, 0.0, 0.0), headlight=True,
                        color=(1.0, 1.0, 1.0), clip_lo=(-1e30, -1e30, -1e30),
                        clip_hi=(1e30, 1e30, 1e30)) -> SurfaceParams:
    g = GRAD[grad] if isinstance(grad, str) else int(grad)
    return SurfaceParams(float(step), float(iso_lo), float(iso_hi), int(refine), g, ka, kd, ks,
                         shininess, (C.c_double * 3)(*light), int(bool(headlight)),
                         (C.c_double * 3)(*color), (C.c_float * 3)(*clip_lo),
                         (C.c_float * 3)(*clip_hi))


def sample_f32(ov: OracleVolume, p) -> float:
    """FP32 trilinear value in raw units (the inside test of the first-hit renderer)."""
    pf = (C.c_float * 3)(*[float(v) for v in p])
    return float(lib().vro_sample_f32(C.byref(ov.s), pf))


def render_surface(ov: OracleVolume, cam: dict, sp: SurfaceParams, rows=None, nthreads=0):
    """First-hit renderer (§3.11 threshold window, §5.1 refinement): returns (rgba (H, W, 4)
    float64, depth (H, W) float32, coarse samples)."""
    H, W = cam["height"], cam["width"]
    r0, r1 = (0, H) if rows is None else rows
    img = np.zeros((H, W, 4), np.float64)
    depth = np.full((H, W), np.inf, np.float32)
    c = make_camera(cam)
    n = lib().vro_render_surface(C.byref(ov.s), C.byref(c), C.byref(sp), _dptr(img),
                                 depth.ctypes.data_as(C.POINTER(C.c_float)), r0, r1, nthreads)
    return img, depth, int(n)
