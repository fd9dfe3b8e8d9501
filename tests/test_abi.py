"""Host-only checks of the C-ABI library: it builds for sm_103a, loads, exports every
entry point declared in include/vr.h, and rejects bad arguments before touching a GPU."""
import ctypes as C
import os
import re

import pytest

from _util import gpu_available

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(vr_[a-z0-9_]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libvr():
    from paper_1609_01317_gb300 import build, vr

    build.build()
    return vr.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vr_create", "vr_destroy", "vr_upload_volume", "vr_set_transfer_function",
                 "vr_set_camera", "vr_render", "vr_render_forward_train", "vr_render_backward",
                 "vr_checkpoint_bytes", "vr_read_stats", "vr_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(libvr):
    for name in declared_functions():
        assert hasattr(libvr, name), name


def test_status_strings(libvr):
    from paper_1609_01317_gb300 import vr

    for code in range(7):
        assert vr.vr_status_string(code) not in ("", "unknown status")
    assert vr.vr_status_string(99) == "unknown status"
    assert vr.vr_version() >= 100


def test_null_arguments_are_rejected_without_a_device(libvr):
    from paper_1609_01317_gb300 import vr

    L = libvr
    assert L.vr_create(None, 0, vr.ALLOC_FN(), vr.FREE_FN(), None) == 1
    h = C.c_void_p()
    # exactly one of alloc / free given
    assert L.vr_create(C.byref(h), 0, vr.ALLOC_FN(lambda n, u: None), vr.FREE_FN(), None) == 1
    assert L.vr_upload_volume(None, None, 0, 1, 1, 1, 1.0, None) == 1
    assert L.vr_set_transfer_function(None, None, 2, None) == 1
    assert L.vr_set_camera(None, None) == 1
    p = vr.make_params()
    assert L.vr_render(None, C.byref(p), None, None) == 1
    assert L.vr_render_rgba8(None, C.byref(p), None, None) == 1
    assert L.vr_render_backward(None, C.byref(p), None, None, None, None, None) == 1
    assert L.vr_read_stats(None, None, None) == 1
    pk = vr.vr_peaks()
    assert L.vr_measure_peaks(0, 5, None) == 1
    assert L.vr_measure_peaks(0, 0, C.byref(pk)) == 1
    assert L.vr_measure_peaks(-1, 5, C.byref(pk)) == 1
    cnt = C.c_ulonglong(7)
    assert L.vr_read_bounds_violations(None, C.byref(cnt), None) == 1
    assert L.vr_probe_samples(None, C.byref(p), None, 1, None, None) == 1
    L.vr_destroy(None)  # no-op


@pytest.mark.skipif(gpu_available(), reason="checks the no-device path")
def test_create_without_a_device_reports_cuda_error(libvr):
    from paper_1609_01317_gb300 import vr

    h = C.c_void_p()
    st = libvr.vr_create(C.byref(h), 0, vr.ALLOC_FN(), vr.FREE_FN(), None)
    assert st in (1, 3)  # no device: invalid ordinal or CUDA error, never OK
    assert h.value is None


def test_renderer_refuses_to_run_without_cuda():
    if gpu_available():
        pytest.skip("a GPU is present")
    from paper_1609_01317_gb300 import Renderer

    with pytest.raises(RuntimeError):
        Renderer(0)


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: with the library absent every call raises."""
    import subprocess
    import sys

    env = dict(os.environ, VR_LIBRARY=str(tmp_path / "absent_libvr.so"))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1609_01317_gb300 import vr\n"
            "try:\n    vr.vr_version()\nexcept RuntimeError as e:\n    print('raised', e)\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and "raised" in r.stdout and "missing" in r.stdout


def test_binding_checks_buffers_before_calling_the_library(libvr):
    """The binding rejects a non-contiguous, short, wrongly typed or host-resident buffer
    with VR_ERR_INVALID_ARG before the library (or a GPU) is touched."""
    import numpy as np
    import torch

    from paper_1609_01317_gb300 import vr

    cam = {"eye": [0, 0, 40], "target": [0, 0, 0], "up": [0, 1, 0], "ortho": 0,
           "fov_y_deg": 40.0, "ortho_height": 1.0, "width": 8, "height": 6}
    p = vr.make_params()

    def rejected(fn, *a):
        with pytest.raises(vr.VrError) as e:
            fn(*a)
        assert e.value.status == 1

    # transposed (non-contiguous) image
    rejected(vr.vr_render, None, p, torch.zeros(6, 8, 4).transpose(0, 1))
    # the 8-bit image takes 1-byte elements
    rejected(vr.vr_render_rgba8, None, p, torch.zeros(6, 8, 4))
    # voxels: too few bytes for 4 x 4 x 4 u16, and u16 voxels given as float32
    rejected(vr.vr_upload_volume, None, np.zeros(60, np.uint16), "u16", 4, 4, 4, 4095.0)
    rejected(vr.vr_upload_volume, None, np.zeros(64, np.float32), "u16", 4, 4, 4, 4095.0)
    # transfer function shorter than n entries
    rejected(vr.vr_set_transfer_function, None, np.zeros((3, 4), np.float32), 4)
    # the allocation-free render takes device memory only, and whole images
    rejected(vr.vr_render_noalloc, np.zeros(64, np.uint8), "u8", 4, 4, 4, 255.0,
             np.zeros((2, 4), np.float32), 2, cam, p, np.zeros((6, 8, 4), np.float32))
    # probe points: 3 floats per point
    rejected(vr.vr_probe_samples, None, p, torch.zeros(5), 2, torch.zeros(24))
