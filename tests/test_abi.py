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
