"""Thin ctypes binding of ``libvr.so`` (the C ABI in ``include/vr.h``).

Argument marshalling only: every step of the ray march runs in the CUDA kernels of the
library.  Functions keep the C names; each raises ``VrError`` on a non-zero status.
Loading fails loudly if the library has not been built (``build.py``); there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# VR_LIBRARY selects another build of the library (the bounds-checked libvr_bounds.so)
LIB_PATH = os.environ.get("VR_LIBRARY") or os.path.join(HERE, "libvr.so")

VR_OK = 0
STATUS_NAMES = {0: "VR_OK", 1: "VR_ERR_INVALID_ARG", 2: "VR_ERR_OUT_OF_MEMORY", 3: "VR_ERR_CUDA",
                4: "VR_ERR_UNSUPPORTED", 5: "VR_ERR_TIMEOUT", 6: "VR_ERR_STATE"}
DTYPES = {"u8": 0, "u16": 1, "f16": 2, "f32": 3}
GRADS = {"central": 0, "sobel3d": 1, "zucker_hummel": 2}


class VrError(RuntimeError):
    def __init__(self, func, status, detail=""):
        self.status = status
        name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{func}: {name}{(' (' + detail + ')') if detail else ''}")


class vr_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("ortho", C.c_int), ("fov_y_deg", C.c_float), ("ortho_height", C.c_float),
                ("width", C.c_int), ("height", C.c_int)]


class vr_render_params(C.Structure):
    _fields_ = [("step", C.c_float), ("grad", C.c_int), ("ka", C.c_float), ("kd", C.c_float),
                ("ks", C.c_float), ("shininess", C.c_float), ("light", C.c_float * 3),
                ("headlight", C.c_int), ("ert_threshold", C.c_float), ("skip_empty", C.c_int),
                ("clip_lo", C.c_float * 3), ("clip_hi", C.c_float * 3),
                ("collect_stats", C.c_int), ("adaptive", C.c_int),
                ("adapt_range2", C.c_float), ("adapt_range4", C.c_float), ("march", C.c_int)]


class vr_surface_params(C.Structure):
    _fields_ = [("step", C.c_float), ("iso_lo", C.c_float), ("iso_hi", C.c_float),
                ("refine", C.c_int), ("grad", C.c_int), ("ka", C.c_float), ("kd", C.c_float),
                ("ks", C.c_float), ("shininess", C.c_float), ("light", C.c_float * 3),
                ("headlight", C.c_int), ("color", C.c_float * 3), ("skip_empty", C.c_int),
                ("clip_lo", C.c_float * 3), ("clip_hi", C.c_float * 3)]


class vr_stats(C.Structure):
    _fields_ = [("rays_hit", C.c_ulonglong), ("samples_plain", C.c_ulonglong),
                ("samples_visited", C.c_ulonglong), ("samples_shaded", C.c_ulonglong),
                ("march", C.c_ulonglong)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("vr_create", C.c_int, [C.POINTER(C.c_void_p), C.c_int, ALLOC_FN, FREE_FN, C.c_void_p]),
    ("vr_destroy", None, [C.c_void_p]),
    ("vr_upload_volume", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.c_float, C.c_void_p]),
    ("vr_set_transfer_function", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    ("vr_set_camera", C.c_int, [C.c_void_p, C.POINTER(vr_camera)]),
    ("vr_render", C.c_int, [C.c_void_p, C.POINTER(vr_render_params), C.c_void_p, C.c_void_p]),
    ("vr_render_rgba8", C.c_int, [C.c_void_p, C.POINTER(vr_render_params), C.c_void_p,
                                  C.c_void_p]),
    ("vr_render_rows", C.c_int, [C.c_void_p, C.POINTER(vr_render_params), C.c_int, C.c_int,
                                 C.c_void_p, C.c_void_p]),
    ("vr_render_partial", C.c_int, [C.c_void_p, C.POINTER(vr_render_params), C.c_float,
                                    C.c_float, C.c_void_p, C.c_void_p]),
    ("vr_checkpoint_bytes", C.c_int, [C.c_void_p, C.POINTER(vr_render_params),
                                      C.POINTER(C.c_size_t)]),
    ("vr_render_forward_train", C.c_int, [C.c_void_p, C.POINTER(vr_render_params), C.c_void_p,
                                          C.c_void_p, C.c_size_t, C.c_void_p]),
    ("vr_render_backward", C.c_int, [C.c_void_p, C.POINTER(vr_render_params), C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("vr_read_stats", C.c_int, [C.c_void_p, C.POINTER(vr_stats), C.c_void_p]),
    ("vr_render_backward_views", C.c_int, [C.c_void_p, C.POINTER(vr_render_params), C.c_int,
                                           C.POINTER(vr_camera), C.POINTER(C.c_void_p),
                                           C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p,
                                           C.c_void_p]),
    ("vr_render_noalloc", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                                    C.c_void_p, C.c_int, C.POINTER(vr_camera),
                                    C.POINTER(vr_render_params), C.c_void_p, C.c_void_p]),
    ("vr_batch_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                                  C.POINTER(vr_camera), C.POINTER(C.c_int), C.c_int,
                                  C.POINTER(vr_render_params), C.POINTER(C.c_void_p),
                                  C.c_void_p]),
    ("vr_batch_run", C.c_int, [C.c_void_p, C.c_void_p]),
    ("vr_batch_autotune", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    ("vr_batch_destroy", None, [C.c_void_p]),
    ("vr_render_surface", C.c_int, [C.c_void_p, C.POINTER(vr_surface_params), C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    ("vr_render_batch", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(vr_camera), C.POINTER(C.c_int),
                                  C.c_int, C.POINTER(vr_render_params), C.POINTER(C.c_void_p),
                                  C.c_void_p]),
    ("vr_probe_samples", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                   C.c_void_p]),
    ("vr_measure_peaks", C.c_int, [C.c_int, C.c_int, C.c_void_p]),
    ("vr_screen_rect", C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                 C.POINTER(C.c_int)]),
    ("vr_read_bounds_violations", C.c_int, [C.c_void_p, C.POINTER(C.c_ulonglong), C.c_void_p]),
    ("vr_status_string", C.c_char_p, [C.c_int]),
    ("vr_last_cuda_error", C.c_char_p, []),
    ("vr_version", C.c_int, []),
]

_lib = None


def lib():
    """Load libvr.so (raises if it is missing: build it with ``build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1609_01317_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(func, status):
    if status != VR_OK:
        detail = ""
        if status == 3:
            detail = lib().vr_last_cuda_error().decode()
        raise VrError(func, status, detail)


def _ptr(x):
    """Address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


# ------------------------------------------------------------- buffer checks
# What the binding knows of each context (image size of the camera, voxel count, table
# entries), so that buffers handed to a call can be checked against what the call touches.
_state = {}
_ELEM = {0: 1, 1: 2, 2: 2, 3: 4}  # bytes per voxel of each vr_dtype


def _buf(func, x, nbytes, elem=None, device_only=False, what="buffer"):
    """Check a torch tensor or numpy array handed to `func`: contiguous, at least `nbytes`
    long, elements of `elem` bytes (when given) and, for `device_only` arguments, CUDA
    memory.  Raises VrError(VR_ERR_INVALID_ARG) before the library is called.  Raw integer
    addresses and None pass unchecked (the library validates what it can)."""
    if x is None or isinstance(x, int):
        return
    if hasattr(x, "data_ptr") and hasattr(x, "is_contiguous"):
        if not x.is_contiguous():
            raise VrError(func, 1, f"{what} is not contiguous")
        if device_only and not x.is_cuda:
            raise VrError(func, 1, f"{what} must be CUDA device memory")
        es, have = x.element_size(), x.numel() * x.element_size()
    elif hasattr(x, "ctypes") and hasattr(x, "flags"):
        if not x.flags["C_CONTIGUOUS"]:
            raise VrError(func, 1, f"{what} is not C-contiguous")
        if device_only:
            raise VrError(func, 1, f"{what} must be CUDA device memory, not a numpy array")
        es, have = x.itemsize, x.nbytes
    else:
        return
    if elem is not None and es != elem:
        raise VrError(func, 1, f"{what} has {es}-byte elements, {elem} expected")
    if have < nbytes:
        raise VrError(func, 1, f"{what} holds {have} bytes, the call touches {nbytes}")


def _image_bytes(cam) -> int:
    if isinstance(cam, vr_camera):
        return int(cam.width) * int(cam.height) * 16
    return int(cam["width"]) * int(cam["height"]) * 16


def make_camera(cam: dict) -> vr_camera:
    return vr_camera((C.c_float * 3)(*cam["eye"]), (C.c_float * 3)(*cam["target"]),
                     (C.c_float * 3)(*cam["up"]), int(bool(cam["ortho"])),
                     float(cam["fov_y_deg"]), float(cam["ortho_height"]), int(cam["width"]),
                     int(cam["height"]))


MARCHES = {"auto": 0, "records": 1, "slabs": 2}


def make_params(step=0.5, grad="central", ka=0.1, kd=0.7, ks=0.2, shininess=20.0,
                light=(0.0, 0.0, 0.0), headlight=True, ert_threshold=0.99, skip_empty=True,
                clip_lo=(-1e30, -1e30, -1e30), clip_hi=(1e30, 1e30, 1e30),
                collect_stats=False, adapt_range=None, march="auto") -> vr_render_params:
    """adapt_range = (bound of multiplier 2, bound of multiplier 4) in raw value units turns
    adaptive sampling on (a negative bound disables its level); None = off.  march: "auto",
    "records" or "slabs" (the kernel a plain render runs; the same image either way)."""
    g = GRADS[grad] if isinstance(grad, str) else int(grad)
    ad = adapt_range is not None
    r2, r4 = (float(adapt_range[0]), float(adapt_range[1])) if ad else (-1.0, -1.0)
    return vr_render_params(float(step), g, float(ka), float(kd), float(ks), float(shininess),
                            (C.c_float * 3)(*light), int(bool(headlight)), float(ert_threshold),
                            int(bool(skip_empty)), (C.c_float * 3)(*clip_lo),
                            (C.c_float * 3)(*clip_hi), int(bool(collect_stats)), int(ad), r2, r4,
                            MARCHES[march] if isinstance(march, str) else int(march))


def make_surface_params(step=2.0, iso_lo=0.5, iso_hi=3.0e38, refine=6, grad="central", ka=0.1,
                        kd=0.7, ks=0.2, shininess=20.0, light=(0.0, 0.0, 0.0), headlight=True,
                        color=(1.0, 1.0, 1.0), skip_empty=True, clip_lo=(-1e30, -1e30, -1e30),
                        clip_hi=(1e30, 1e30, 1e30)) -> vr_surface_params:
    g = GRADS[grad] if isinstance(grad, str) else int(grad)
    return vr_surface_params(float(step), float(iso_lo), float(iso_hi), int(refine), g, float(ka),
                             float(kd), float(ks), float(shininess), (C.c_float * 3)(*light),
                             int(bool(headlight)), (C.c_float * 3)(*color), int(bool(skip_empty)),
                             (C.c_float * 3)(*clip_lo), (C.c_float * 3)(*clip_hi))


# ----------------------------------------------------------- same-name wrappers
def vr_create(device=0, alloc=None, free=None, user=None):
    h = C.c_void_p()
    a = alloc if alloc is not None else ALLOC_FN()
    f = free if free is not None else FREE_FN()
    _check("vr_create", lib().vr_create(C.byref(h), int(device), a, f, user))
    _state[h.value] = {}
    return h.value


def vr_destroy(ctx):
    _state.pop(ctx, None)
    lib().vr_destroy(ctx)


def vr_upload_volume(ctx, voxels, dtype, nx, ny, nz, value_max, stream=None):
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    nvox = int(nx) * int(ny) * int(nz)
    _buf("vr_upload_volume", voxels, nvox * _ELEM.get(dt, 1), _ELEM.get(dt), what="voxels")
    _check("vr_upload_volume", lib().vr_upload_volume(ctx, _ptr(voxels), dt, int(nx), int(ny),
                                                      int(nz), float(value_max), stream))
    _state.setdefault(ctx, {})["nvox"] = nvox


def vr_set_transfer_function(ctx, rgba, n, stream=None):
    _buf("vr_set_transfer_function", rgba, int(n) * 16, 4, what="rgba")
    _check("vr_set_transfer_function", lib().vr_set_transfer_function(ctx, _ptr(rgba), int(n),
                                                                      stream))
    _state.setdefault(ctx, {})["ntf"] = int(n)


def vr_set_camera(ctx, cam):
    c = cam if isinstance(cam, vr_camera) else make_camera(cam)
    _check("vr_set_camera", lib().vr_set_camera(ctx, C.byref(c)))
    _state.setdefault(ctx, {})["image"] = _image_bytes(c)
    _state[ctx]["height"] = int(c.height)


def vr_render(ctx, params, out_rgba, stream=None):
    _buf("vr_render", out_rgba, _state.get(ctx, {}).get("image", 0), 4, what="out_rgba")
    _check("vr_render", lib().vr_render(ctx, C.byref(params), _ptr(out_rgba), stream))


def vr_render_rgba8(ctx, params, out_rgba8, stream=None):
    """vr_render's image with 8 bits per channel into an H x W x 4 byte buffer."""
    _buf("vr_render_rgba8", out_rgba8, _state.get(ctx, {}).get("image", 0) // 4, 1,
         what="out_rgba8")
    _check("vr_render_rgba8", lib().vr_render_rgba8(ctx, C.byref(params), _ptr(out_rgba8),
                                                    stream))


def vr_render_rows(ctx, params, row0, row1, out_rgba, stream=None):
    """Rows [row0, row1) of vr_render's image into a (row1 - row0) x W x 4 band."""
    img = _state.get(ctx, {}).get("image", 0)
    H = _state.get(ctx, {}).get("height", 0)
    band = img // H * (int(row1) - int(row0)) if H and row1 > row0 else 0
    _buf("vr_render_rows", out_rgba, band, 4, what="out_rgba")
    _check("vr_render_rows", lib().vr_render_rows(ctx, C.byref(params), int(row0), int(row1),
                                                  _ptr(out_rgba), stream))


def vr_render_partial(ctx, params, z0, z1, out_rgba, stream=None):
    """The premultiplied partial image of the samples with z in [z0, z1) (sort-last)."""
    _buf("vr_render_partial", out_rgba, _state.get(ctx, {}).get("image", 0), 4, what="out_rgba")
    _check("vr_render_partial", lib().vr_render_partial(ctx, C.byref(params), float(z0),
                                                        float(z1), _ptr(out_rgba), stream))


def vr_checkpoint_bytes(ctx, params) -> int:
    n = C.c_size_t()
    _check("vr_checkpoint_bytes", lib().vr_checkpoint_bytes(ctx, C.byref(params), C.byref(n)))
    return n.value


def vr_render_forward_train(ctx, params, out_rgba, checkpoints, checkpoint_bytes, stream=None):
    _buf("vr_render_forward_train", out_rgba, _state.get(ctx, {}).get("image", 0), 4, True,
         "out_rgba")
    _buf("vr_render_forward_train", checkpoints, int(checkpoint_bytes), None, True, "checkpoints")
    _check("vr_render_forward_train",
           lib().vr_render_forward_train(ctx, C.byref(params), _ptr(out_rgba), _ptr(checkpoints),
                                         int(checkpoint_bytes), stream))


def vr_render_backward(ctx, params, checkpoints, grad_rgba, grad_volume, grad_tf, stream=None):
    st = _state.get(ctx, {})
    _buf("vr_render_backward", grad_rgba, st.get("image", 0), 4, True, "grad_rgba")
    _buf("vr_render_backward", grad_volume, 4 * st.get("nvox", 0), 4, True, "grad_volume")
    _buf("vr_render_backward", grad_tf, 16 * st.get("ntf", 0), 4, True, "grad_tf")
    _check("vr_render_backward",
           lib().vr_render_backward(ctx, C.byref(params), _ptr(checkpoints), _ptr(grad_rgba),
                                    _ptr(grad_volume), _ptr(grad_tf), stream))


def vr_render_noalloc(voxels, dtype, nx, ny, nz, value_max, tf_rgba, ntf, cam, params,
                      out_rgba, stream=None):
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    c = cam if isinstance(cam, vr_camera) else make_camera(cam)
    f = "vr_render_noalloc"
    _buf(f, voxels, int(nx) * int(ny) * int(nz) * _ELEM.get(dt, 1), _ELEM.get(dt), True, "voxels")
    _buf(f, tf_rgba, int(ntf) * 16, 4, True, "tf_rgba")
    _buf(f, out_rgba, _image_bytes(c), 4, True, "out_rgba")
    _check("vr_render_noalloc",
           lib().vr_render_noalloc(_ptr(voxels), dt, int(nx), int(ny), int(nz), float(value_max),
                                   _ptr(tf_rgba), int(ntf), C.byref(c), C.byref(params),
                                   _ptr(out_rgba), stream))


def vr_render_backward_views(ctx, params, cams, checkpoints, grad_rgbas, grad_volume, grad_tf,
                             stream=None):
    n = len(cams)
    carr = (vr_camera * n)(*[c if isinstance(c, vr_camera) else make_camera(c) for c in cams])
    st = _state.get(ctx, {})
    for c, g in zip(carr, grad_rgbas):
        _buf("vr_render_backward_views", g, _image_bytes(c), 4, True, "grad_rgba")
    _buf("vr_render_backward_views", grad_volume, 4 * st.get("nvox", 0), 4, True, "grad_volume")
    _buf("vr_render_backward_views", grad_tf, 16 * st.get("ntf", 0), 4, True, "grad_tf")
    karr = (C.c_void_p * n)(*[_ptr(k) for k in checkpoints])
    garr = (C.c_void_p * n)(*[_ptr(g) for g in grad_rgbas])
    _check("vr_render_backward_views",
           lib().vr_render_backward_views(ctx, C.byref(params), n, carr, karr, garr,
                                          _ptr(grad_volume), _ptr(grad_tf), stream))


def vr_read_stats(ctx, stream=None) -> dict:
    s = vr_stats()
    _check("vr_read_stats", lib().vr_read_stats(ctx, C.byref(s), stream))
    return {k: getattr(s, k) for k, _ in vr_stats._fields_}


def vr_batch_create(ctxs, cams, ctx_of_cam, params, outs, stream=None):
    n = len(cams)
    h = C.c_void_p()
    carr = (C.c_void_p * len(ctxs))(*ctxs)
    cams_arr = (vr_camera * n)(*[c if isinstance(c, vr_camera) else make_camera(c) for c in cams])
    for c, o in zip(cams_arr, outs):
        _buf("vr_batch_create", o, _image_bytes(c), 4, True, "outs[i]")
    idx = (C.c_int * n)(*[int(i) for i in ctx_of_cam])
    oarr = (C.c_void_p * n)(*[_ptr(o) for o in outs])
    _check("vr_batch_create", lib().vr_batch_create(C.byref(h), carr, len(ctxs), cams_arr, idx, n,
                                                    C.byref(params), oarr, stream))
    return h.value


def vr_batch_run(batch, stream=None):
    _check("vr_batch_run", lib().vr_batch_run(batch, stream))


def vr_batch_autotune(batch, stream=None):
    ch = (C.c_int * 3)()
    _check("vr_batch_autotune", lib().vr_batch_autotune(batch, stream, ch))
    return tuple(ch)


def vr_batch_destroy(batch):
    lib().vr_batch_destroy(batch)


def vr_render_surface(ctx, params, out_rgba, out_depth=None, stream=None):
    img = _state.get(ctx, {}).get("image", 0)
    _buf("vr_render_surface", out_rgba, img, 4, what="out_rgba")
    _buf("vr_render_surface", out_depth, img // 4, 4, what="out_depth")
    _check("vr_render_surface", lib().vr_render_surface(ctx, C.byref(params), _ptr(out_rgba),
                                                        _ptr(out_depth), stream))


def vr_render_batch(vols, cams, vol_of_cam, params, outs, stream=None):
    n = len(cams)
    varr = (C.c_void_p * len(vols))(*vols)
    cams_arr = (vr_camera * n)(*[c if isinstance(c, vr_camera) else make_camera(c) for c in cams])
    for c, o in zip(cams_arr, outs):
        _buf("vr_render_batch", o, _image_bytes(c), 4, True, "outs[i]")
    idx = (C.c_int * n)(*[int(i) for i in vol_of_cam])
    oarr = (C.c_void_p * n)(*[_ptr(o) for o in outs])
    _check("vr_render_batch", lib().vr_render_batch(varr, cams_arr, idx, n, C.byref(params), oarr,
                                                    stream))


def vr_screen_rect(cam, lo, hi):
    """(x0, y0, x1, y1): pixels outside [x0, x1) x [y0, y1) see nothing of the box [lo, hi]."""
    c = cam if isinstance(cam, vr_camera) else make_camera(cam)
    r = (C.c_int * 4)()
    _check("vr_screen_rect", lib().vr_screen_rect(C.byref(c), (C.c_float * 3)(*lo),
                                                  (C.c_float * 3)(*hi), r))
    return tuple(r)


def vr_probe_samples(ctx, params, pos, n, out, stream=None):
    _buf("vr_probe_samples", pos, 12 * max(int(n), 0), 4, True, "pos")
    _buf("vr_probe_samples", out, 48 * max(int(n), 0), 4, True, "out")
    _check("vr_probe_samples", lib().vr_probe_samples(ctx, C.byref(params), _ptr(pos), int(n),
                                                      _ptr(out), stream))


def vr_read_bounds_violations(ctx, stream=None) -> int:
    n = C.c_ulonglong(0)
    _check("vr_read_bounds_violations", lib().vr_read_bounds_violations(ctx, C.byref(n), stream))
    return int(n.value)


class vr_peaks(C.Structure):
    _fields_ = [("fma_tflops", C.c_double), ("gather_coherent_gsps", C.c_double),
                ("gather_random_gsps", C.c_double), ("gather_u16_random_gsps", C.c_double),
                ("gather_u16_coherent_gsps", C.c_double)]


def vr_measure_peaks(device=0, repeats=5) -> dict:
    p = vr_peaks()
    _check("vr_measure_peaks", lib().vr_measure_peaks(int(device), int(repeats), C.byref(p)))
    return {k: getattr(p, k) for k, _ in vr_peaks._fields_}


def vr_status_string(status) -> str:
    return lib().vr_status_string(int(status)).decode()


def vr_version() -> int:
    return lib().vr_version()
