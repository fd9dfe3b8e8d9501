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


def _noalloc(vol, dt, vmax, tf, cam, params):
    import torch
    from paper_1609_01317_gb300 import vr

    host = vol.view(np.int16) if vol.dtype == np.uint16 else vol
    vdev = torch.from_numpy(np.ascontiguousarray(host)).cuda()
    tdev = torch.from_numpy(tf).cuda()
    out = torch.full((cam["height"], cam["width"], 4), float("nan"), device="cuda")
    nz, ny, nx = vol.shape
    vr.vr_render_noalloc(vdev, dt, nx, ny, nz, vmax, tdev, tf.shape[0], cam, params, out,
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("case", ["u8_central", "f16_zucker_hummel", "u16_sobel_thin_x",
                                  "f32_central_thin_z"])
def test_noalloc_render_matches_the_oracle(case):
    """Every voxel type and operator of the allocation-free render against the FP64 oracle
    (§3.10), including volumes two voxels thick along x and along z (every cell index
    clamps to 0 there), each rendered twice in a row through the shared scratch array."""
    import oracle
    from paper_1609_01317_gb300 import build, vr

    build.build()
    if case == "u8_central":
        vol, dt, vmax, grad = P.sphere_u8(0, 24, 9.0), "u8", 255.0, "central"
        tf = P.tf_c1(256)
    elif case == "f16_zucker_hummel":
        vol = (P.ellipsoids(3, (28, 22, 19), count=5).astype(np.float32) / 4095.0).astype(np.float16)
        dt, vmax, grad, tf = "f16", 1.0, "zucker_hummel", P.tf_two_plateau(256)
    elif case == "u16_sobel_thin_x":
        vol, dt, vmax, grad = P.ellipsoids(4, (2, 21, 17), count=4), "u16", 4095.0, "sobel3d"
        tf = P.tf_two_plateau(256)
    else:
        vol = P.random_volume(5, (13, 11, 2), np.float32, 1.0)
        dt, vmax, grad, tf = "f32", 1.0, "central", P.tf_random(6, 64, alpha_max=0.3)
    nz, ny, nx = vol.shape
    cam = P.orbit_camera((nx, ny, nz), 64, 48, 0.9, 0.3, 40.0, radius_diag=1.6)
    for skip in (True, False):
        params = vr.make_params(grad=grad, skip_empty=skip)
        a1 = _noalloc(vol, dt, vmax, tf, cam, params)
        a2 = _noalloc(vol, dt, vmax, tf, cam, params)
        ref, counts, _ = oracle.render(oracle.OracleVolume(vol, vmax), tf, cam,
                                       oracle.make_params(grad=grad))
        assert (counts > 0).sum() > 50
        assert np.isfinite(a1).all()
        assert np.array_equal(a1, a2)  # the second call sees the first call's scratch
        assert_image_parity(a1, ref, f"noalloc {case} skip {skip}")


def test_noalloc_rejects_misaligned_pointers_before_any_work():
    """The kernels read the table and write the image as float4 and read voxels as whole
    elements: misaligned addresses are refused on the host (nothing is launched, so the
    output keeps its contents)."""
    import torch
    from paper_1609_01317_gb300 import vr

    cam = P.orbit_camera((8, 8, 8), 8, 8, 0.1, 0.2, 40.0)
    p = vr.make_params()
    tf = torch.rand((9, 4), device="cuda")
    out = torch.full((8 * 8 * 4 + 4,), 7.0, device="cuda")
    vol = torch.zeros(8 * 8 * 8 + 2, device="cuda", dtype=torch.int16)
    good_out, bad_out = out.data_ptr(), out.data_ptr() + 4
    cases = [(vol.data_ptr() + 1, "u16", tf.data_ptr(), good_out),  # voxels off by one byte
             (vol.data_ptr(), "u16", tf.data_ptr() + 4, good_out),  # table off by 4 bytes
             (vol.data_ptr(), "u16", tf.data_ptr(), bad_out)]       # image off by 4 bytes
    for v, dt, t, o in cases:
        with pytest.raises(vr.VrError) as e:
            vr.vr_render_noalloc(v, dt, 8, 8, 8, 4095.0, t, 8, cam, p, o)
        assert e.value.status == 1
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
