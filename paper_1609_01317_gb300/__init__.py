"""GB300-native direct volume ray caster (method of "Volume Raycasting mit OpenCL",
Kopal 2011, arXiv:1609.01317).

The compute path is the CUDA library ``libvr.so`` behind the C ABI of ``include/vr.h``;
``vr`` is its ctypes binding (same names as the C entry points).  ``Renderer`` wraps a
context for PyTorch users: device memory comes from PyTorch's caching allocator, work is
queued on PyTorch's current CUDA stream, and ``render_differentiable`` exposes the
adjoint kernel as a ``torch.autograd.Function``.  There is no CPU fallback: without a
built library or a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes as C

from . import vr

__all__ = ["vr", "Renderer", "render_differentiable"]

_TORCH_DTYPES = {"u8": "uint8", "u16": "uint16", "f16": "float16", "f32": "float32"}


def _torch():
    import torch

    return torch


def _stream_handle():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream or None


def _dtype_name(t) -> str:
    torch = _torch()
    m = {torch.uint8: "u8", torch.float16: "f16", torch.float32: "f32"}
    if hasattr(torch, "uint16"):
        m[torch.uint16] = "u16"
    if t.dtype in m:
        return m[t.dtype]
    if t.dtype == torch.int16:
        return "u16"  # reinterpreted bit pattern (12-bit values are non-negative)
    raise TypeError(f"unsupported voxel dtype {t.dtype}")


class Renderer:
    """One libvr context on one CUDA device.

    Volumes are torch tensors (or numpy arrays) of shape (nz, ny, nx), x fastest, dtype
    uint8 / uint16 (or int16 holding 12-bit values) / float16 / float32.
    """

    def __init__(self, device: int = 0, use_torch_allocator: bool = True):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("libvr needs a CUDA device; no CPU fallback exists")
        self.device = int(device)
        self._keep = []
        if use_torch_allocator:
            dev = self.device

            def _alloc(nbytes, user):
                try:
                    with torch.cuda.device(dev):
                        return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
                except Exception:  # out of memory -> NULL -> VR_ERR_OUT_OF_MEMORY
                    return None

            def _free(ptr, user):
                with torch.cuda.device(dev):
                    torch.cuda.caching_allocator_delete(ptr)

            a, f = vr.ALLOC_FN(_alloc), vr.FREE_FN(_free)
            self._keep += [a, f]
            self.ctx = vr.vr_create(self.device, a, f)
        else:
            self.ctx = vr.vr_create(self.device)
        self.shape_xyz = None
        self.value_max = None
        self.ntf = None
        self.camera = None

    def close(self):
        if getattr(self, "ctx", None):
            vr.vr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- state
    def upload_volume(self, volume, value_max: float, dtype: str | None = None):
        """Upload a (nz, ny, nx) volume from host (numpy / CPU tensor) or device memory."""
        torch = _torch()
        self._vol_key = None
        if hasattr(volume, "dtype") and isinstance(volume, torch.Tensor):
            t = volume.contiguous()
            name = dtype or _dtype_name(t)
            self._vol_ref = t
        else:
            import numpy as np

            a = np.ascontiguousarray(volume)
            name = dtype or {np.dtype(np.uint8): "u8", np.dtype(np.uint16): "u16",
                             np.dtype(np.float16): "f16", np.dtype(np.float32): "f32"}[a.dtype]
            self._vol_ref = a
        nz, ny, nx = volume.shape
        vr.vr_upload_volume(self.ctx, self._vol_ref, name, nx, ny, nz, value_max,
                            _stream_handle())
        self.shape_xyz = (nx, ny, nz)
        self.value_max = float(value_max)
        self.dtype = name

    def set_transfer_function(self, tf):
        """Set an (n, 4) float32 RGBA table from host or device memory."""
        torch = _torch()
        if isinstance(tf, torch.Tensor):
            t = tf.detach().to(torch.float32).contiguous()
        else:
            import numpy as np

            t = np.ascontiguousarray(tf, np.float32)
        self._tf_ref = t
        self._tf_key = None
        vr.vr_set_transfer_function(self.ctx, t, t.shape[0], _stream_handle())
        self.ntf = int(t.shape[0])

    def set_camera(self, cam: dict):
        vr.vr_set_camera(self.ctx, cam)
        self.camera = dict(cam)

    # ---------------------------------------------------------------- render
    def render(self, params=None, out=None, **kw):
        """Render the current state; returns an (H, W, 4) float32 CUDA tensor."""
        torch = _torch()
        p = params if params is not None else vr.make_params(**kw)
        H, W = self.camera["height"], self.camera["width"]
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.float32, device=f"cuda:{self.device}")
        vr.vr_render(self.ctx, p, out, _stream_handle())
        return out

    def render_rgba8(self, params=None, out=None, **kw):
        """``render``'s image with 8 bits per channel (round(255 clamp(c, 0, 1)) of every
        channel) as an (H, W, 4) uint8 CUDA tensor."""
        torch = _torch()
        p = params if params is not None else vr.make_params(**kw)
        H, W = self.camera["height"], self.camera["width"]
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.uint8, device=f"cuda:{self.device}")
        vr.vr_render_rgba8(self.ctx, p, out, _stream_handle())
        return out

    def render_rows(self, row0: int, row1: int, params=None, out=None, **kw):
        """Rows [row0, row1) of ``render``'s image as a (row1 - row0, W, 4) float32 CUDA
        tensor (bit for bit those rows of the whole frame)."""
        torch = _torch()
        p = params if params is not None else vr.make_params(**kw)
        W = self.camera["width"]
        if out is None:
            out = torch.empty((row1 - row0, W, 4), dtype=torch.float32,
                              device=f"cuda:{self.device}")
        vr.vr_render_rows(self.ctx, p, row0, row1, out, _stream_handle())
        return out

    def render_partial(self, z0: float, z1: float, params=None, out=None, **kw):
        """The premultiplied partial image of the samples with z in [z0, z1) (sort-last,
        ``sortlast.py``) as an (H, W, 4) float32 CUDA tensor."""
        torch = _torch()
        p = params if params is not None else vr.make_params(**kw)
        H, W = self.camera["height"], self.camera["width"]
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.float32, device=f"cuda:{self.device}")
        vr.vr_render_partial(self.ctx, p, z0, z1, out, _stream_handle())
        return out

    def render_surface(self, params=None, out=None, depth=None, **kw):
        """First-hit surface render of the current volume and camera (§3.11, §5.1); returns
        ((H, W, 4) float32 image, (H, W) float32 hit distances, +inf where nothing is hit)."""
        torch = _torch()
        p = params if params is not None else vr.make_surface_params(**kw)
        H, W = self.camera["height"], self.camera["width"]
        dev = f"cuda:{self.device}"
        if out is None:
            out = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
        if depth is None:
            depth = torch.empty((H, W), dtype=torch.float32, device=dev)
        vr.vr_render_surface(self.ctx, p, out, depth, _stream_handle())
        return out, depth

    def stats(self) -> dict:
        return vr.vr_read_stats(self.ctx, _stream_handle())

    def checkpoint_bytes(self, params) -> int:
        return vr.vr_checkpoint_bytes(self.ctx, params)


class _RenderFn:
    """Namespace holder for the autograd Function (built lazily so that importing this
    package does not import torch)."""

    fn = None


def _make_autograd():
    torch = _torch()

    class RenderFunction(torch.autograd.Function):
        """Image = render(volume, tf) for one camera; differentiable in both inputs.

        volume: (nz, ny, nx) float32 CUDA tensor (value_max 1: s = voxel value);
        tf: (n, 4) float32 CUDA tensor.  The forward records the adjoint checkpoints in a
        tensor owned by the autograd graph; the backward calls vr_render_backward.
        """

        @staticmethod
        def forward(ctx_, renderer, volume, tf, camera, params):
            volume = volume.detach().contiguous()
            tf = tf.detach().contiguous()
            # upload only what changed, so that the checkpoints of earlier views in the
            # same graph stay valid (an upload invalidates them)
            vkey = (volume.data_ptr(), volume._version, tuple(volume.shape))
            if getattr(renderer, "_vol_key", None) != vkey:
                renderer.upload_volume(volume, 1.0, "f32")
                renderer._vol_key = vkey
            tkey = (tf.data_ptr(), tf._version, tuple(tf.shape))
            if getattr(renderer, "_tf_key", None) != tkey:
                renderer.set_transfer_function(tf)
                renderer._tf_key = tkey
            renderer.set_camera(camera)
            nbytes = renderer.checkpoint_bytes(params)
            ck = torch.empty(nbytes + 256, dtype=torch.uint8, device=volume.device)
            off = (-ck.data_ptr()) % 256
            ckv = ck[off:off + nbytes]
            H, W = camera["height"], camera["width"]
            img = torch.empty((H, W, 4), dtype=torch.float32, device=volume.device)
            vr.vr_render_forward_train(renderer.ctx, params, img, ckv, nbytes, _stream_handle())
            ctx_.save_for_backward(volume, tf, ck)
            ctx_.ckv_off = off
            ctx_.nbytes = nbytes
            ctx_.renderer = renderer
            ctx_.camera = camera
            ctx_.params = params
            return img

        @staticmethod
        def backward(ctx_, grad_img):
            volume, tf, ck = ctx_.saved_tensors
            r = ctx_.renderer
            # re-establish the forward state if other renders happened in between
            if r.camera != ctx_.camera:
                r.set_camera(ctx_.camera)
            g = grad_img.contiguous().to(torch.float32)
            gv = torch.zeros_like(volume) if ctx_.needs_input_grad[1] else None
            gt = torch.zeros_like(tf) if ctx_.needs_input_grad[2] else None
            ckv = ck[ctx_.ckv_off:ctx_.ckv_off + ctx_.nbytes]
            vr.vr_render_backward(r.ctx, ctx_.params, ckv, g, gv, gt, _stream_handle())
            return None, gv, gt, None, None

    return RenderFunction


def render_differentiable(renderer: Renderer, volume, tf, camera: dict, params):
    """Differentiable render of one view (see RenderFunction)."""
    if _RenderFn.fn is None:
        _RenderFn.fn = _make_autograd()
    return _RenderFn.fn.apply(renderer, volume, tf, camera, params)
