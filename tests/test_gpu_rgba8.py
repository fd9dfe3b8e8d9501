"""vr_render_rgba8: vr_render's image with 8 bits per channel.

The bytes must equal vr_render's FP32 image quantised as round(255 clamp(c, 0, 1)) (FP32
product, ties to even) bit for bit, for device and host outputs, and stay within the image
tolerance of the FP64 oracle's image quantised the same way: 2e-3 on >= 99.9 % of the
values (at most one step of 1/255) and 2e-2 on all of them (at most 6 steps)."""
import numpy as np
import pytest

import oracle
import phantoms as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    from paper_1609_01317_gb300 import Renderer, build

    build.build()
    r = Renderer(0)
    yield r
    torch.cuda.synchronize()
    r.close()


def quantize(img):
    """round(255 clamp(c, 0, 1)) per channel with an FP32 product, ties to even."""
    c = np.clip(np.asarray(img, np.float32), np.float32(0.0), np.float32(1.0))
    return np.rint(c * np.float32(255.0)).astype(np.uint8)


def _render_both(R, w, cam):
    import torch
    from paper_1609_01317_gb300 import vr

    R.upload_volume(w["volume"], w["value_max"])
    R.set_transfer_function(w["tf"])
    R.set_camera(cam)
    kw = dict(step=w["step"], grad=w["grad"], skip_empty=w["skip_empty"])
    f32 = R.render(**kw)
    dev8 = R.render_rgba8(**kw)
    host8 = np.full((cam["height"], cam["width"], 4), 7, np.uint8)
    stream = torch.cuda.current_stream().cuda_stream or None
    vr.vr_render_rgba8(R.ctx, vr.make_params(**kw), host8, stream)
    torch.cuda.synchronize()
    return f32.cpu().numpy(), dev8.cpu().numpy(), host8


def _oracle_steps(w, cam, img8):
    ref, _, _ = oracle.render(oracle.OracleVolume(w["volume"], w["value_max"]), w["tf"], cam,
                              oracle.make_params(step=w["step"], grad=w["grad"]))
    return np.abs(img8.astype(np.int32) - quantize(ref).astype(np.int32))


@pytest.mark.parametrize("name", ["sphere64", "ellipsoids96"])
def test_rgba8_is_the_quantised_fp32_image_and_matches_the_oracle(R, name):
    if name == "sphere64":
        w = P.workload_sphere_64()
    else:
        w = P.workload_ellipsoids_256(160, 120, shape=(96, 96, 96))
    cam = w["camera"]
    f32, dev8, host8 = _render_both(R, w, cam)
    assert dev8.dtype == np.uint8 and dev8.shape == (cam["height"], cam["width"], 4)
    want = quantize(f32)
    assert np.array_equal(dev8, want), int(np.abs(dev8.astype(int) - want).max())
    assert np.array_equal(host8, want)
    assert (dev8[..., 3] > 0).sum() > 200  # the object is in view (small ellipsoids: 991 pixels)
    steps = _oracle_steps(w, cam, dev8)
    assert (steps <= 1).mean() >= 0.999 and steps.max() <= 6, (name, steps.max())


def test_rgba8_rejects_a_misaligned_device_buffer_before_any_work(R):
    import torch
    from paper_1609_01317_gb300 import vr

    w = P.workload_sphere_64()
    R.upload_volume(w["volume"], w["value_max"])
    R.set_transfer_function(w["tf"])
    R.set_camera(w["camera"])
    n = w["camera"]["height"] * w["camera"]["width"] * 4
    buf = torch.full((n + 4,), 9, dtype=torch.uint8, device="cuda")
    with pytest.raises(vr.VrError) as e:
        vr.vr_render_rgba8(R.ctx, vr.make_params(step=0.5, grad="central"),
                           buf.data_ptr() + 1, None)
    assert e.value.status == 1
    torch.cuda.synchronize()
    assert bool((buf == 9).all())
