"""vr_render_noalloc: the allocation-free render for callers that cannot allocate device
memory (a plug-in inside an application that owns the whole device pool, a real-time loop
with a fixed budget, a process whose memory another framework has reserved).  Its output
must equal vr_render's on the same inputs, on consecutive calls that reuse the shared
scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

import phantoms as P
from _util import assert_image_parity

pytestmark = pytest.mark.gpu


def _case(seed, shape, grad, dtype="u16"):
    vol = P.ellipsoids(seed, shape, count=5)
    vmax = 4095.0
    if dtype == "f32":
        vol = (vol.astype(np.float32) / 4095.0)
        vmax = 1.0
    tf = P.tf_two_plateau(256)
    cam = P.orbit_camera(shape, 96, 80, 0.3 + seed, 0.25, 40.0)
    return vol, vmax, tf, cam, grad


def test_noalloc_render_matches_context_render_on_consecutive_calls():
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    R = Renderer(0)
    try:
        for seed, shape, grad, dt in ((1, (40, 36, 30), "zucker_hummel", "u16"),
                                      (2, (24, 31, 17), "sobel3d", "f32")):
            vol, vmax, tf, cam, grad = _case(seed, shape, grad, dt)
            for skip in (True, False):
                params = vr.make_params(grad=grad, skip_empty=skip)
                R.upload_volume(vol, vmax)
                R.set_transfer_function(tf)
                R.set_camera(cam)
                ref = R.render(params=params)
                vdev = torch.from_numpy(vol.view(np.int16) if vol.dtype == np.uint16 else vol).cuda()
                tdev = torch.from_numpy(tf).cuda()
                out = torch.full_like(ref, float("nan"))
                nz, ny, nx = vol.shape
                vr.vr_render_noalloc(vdev, "u16" if dt == "u16" else "f32", nx, ny, nz, vmax,
                                     tdev, tf.shape[0], cam, params, out,
                                     torch.cuda.current_stream().cuda_stream)
                torch.cuda.synchronize()
                a, b = out.cpu().numpy(), ref.cpu().numpy()
                assert np.isfinite(a).all()
                assert_image_parity(a, b, f"noalloc seed {seed} skip {skip}")
                assert np.abs(a - b).max() < 1e-4
    finally:
        torch.cuda.synchronize()
        R.close()


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    from paper_1609_01317_gb300 import vr

    cam = P.orbit_camera((8, 8, 8), 8, 8, 0.1, 0.2, 40.0)
    tf = torch.zeros((8, 4), device="cuda")
    out = torch.empty((8, 8, 4), device="cuda")
    vol = torch.zeros(8, device="cuda", dtype=torch.uint8)
    # 4096 x 4096 x 128 voxels = 512 x 512 x 16 = 4 Mi bricks > 262144
    with pytest.raises(vr.VrError) as e:
        vr.vr_render_noalloc(vol, "u8", 4096, 4096, 128, 255.0, tf, 8, cam, vr.make_params(), out)
    assert e.value.status == 1
    with pytest.raises(vr.VrError) as e:  # transfer function beyond 4096 entries
        vr.vr_render_noalloc(vol, "u8", 2, 2, 2, 255.0, tf, 5000, cam, vr.make_params(), out)
    assert e.value.status == 1
    host = np.zeros(8, np.uint8)
    with pytest.raises(vr.VrError):  # host memory is refused
        vr.vr_render_noalloc(host, "u8", 2, 2, 2, 255.0, tf, 8, cam, vr.make_params(), out)
