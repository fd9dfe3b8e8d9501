"""First-hit surface rendering (vr_render_surface) against the FP64 oracle.

The inside / outside decisions are FP32 on both sides with the same operations, so the hit
distances must agree bit for bit; the shaded colour (FP32 on the GPU, FP64 in the oracle)
must meet the image tolerance.
"""
import numpy as np
import pytest

import oracle
import phantoms as P
from _util import assert_image_parity

pytestmark = pytest.mark.gpu


def _gpu_surface(vol, vmax, cam, **kw):
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    r = Renderer(0)
    try:
        r.upload_volume(vol, vmax)
        r.set_camera(cam)
        img, depth = r.render_surface(params=vr.make_surface_params(**kw))
        torch.cuda.synchronize()
        return img.cpu().numpy(), depth.cpu().numpy()
    finally:
        r.close()


def _oracle_surface(vol, vmax, cam, rows=None, **kw):
    kw = dict(kw)
    kw.pop("skip_empty", None)
    ov = oracle.OracleVolume(vol, vmax)
    img, depth, _ = oracle.render_surface(ov, cam, oracle.make_surface_params(**kw), rows=rows)
    return img, depth


def _check(vol, vmax, cam, what, min_hits=50, **kw):
    g_img, g_depth = _gpu_surface(vol, vmax, cam, **kw)
    o_img, o_depth = _oracle_surface(vol, vmax, cam, **kw)
    assert np.array_equal(g_depth, o_depth), (
        f"{what}: depth differs at {np.argwhere(g_depth != o_depth)[:5].tolist()}")
    hits = np.isfinite(o_depth)
    assert hits.sum() >= min_hits, f"{what}: only {hits.sum()} hits"
    assert np.all(g_img[~hits] == 0.0)
    assert np.all(g_img[hits, 3] == 1.0)
    assert_image_parity(g_img, o_img, what)


@pytest.mark.parametrize("dtype,vmax", [(np.uint8, 255.0), (np.uint16, 4095.0),
                                        (np.float16, 1.0), (np.float32, 1.0)])
@pytest.mark.parametrize("grad", ["central", "sobel3d", "zucker_hummel"])
def test_surface_parity_dtypes_and_operators(dtype, vmax, grad):
    shp = (37, 29, 23)  # ragged: not a multiple of the 8^3 bricks
    if dtype in (np.float16, np.float32):
        vol = P.blurred_random_field(21, 40)[:23, :29, :37].astype(dtype)
    else:
        vol = P.ellipsoids(31, shp, value_max=vmax, dtype=dtype)
    lo = float(np.percentile(vol.astype(np.float64), 70))
    for i, cam in enumerate([P.orbit_camera(shp, 41, 33, 0.5, 0.3, 40.0),
                             P.orbit_camera(shp, 40, 32, 2.2, -0.5, 0.0, ortho=True,
                                            ortho_height=50.0)]):
        for refine, skip in ((0, True), (6, True), (6, False)):
            _check(vol, vmax, cam, f"{dtype.__name__} {grad} cam{i} r{refine} skip{skip}",
                   step=1.5, iso_lo=lo, iso_hi=3.0e38, refine=refine, grad=grad,
                   skip_empty=skip, color=(0.9, 0.7, 0.5))


def test_surface_two_sided_window_and_point_light():
    vol = P.ellipsoids(32, (48, 40, 44), value_max=4095.0, dtype=np.uint16)
    lo, hi = np.percentile(vol, [55, 80])
    cam = P.orbit_camera((48, 40, 44), 48, 40, 1.0, 0.6, 40.0)
    _check(vol, 4095.0, cam, "band window, point light", step=2.0, iso_lo=float(lo),
           iso_hi=float(hi), refine=5, grad="sobel3d", headlight=False,
           light=(200.0, -50.0, 120.0))


def test_surface_skipping_never_changes_a_pixel():
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    vol = P.ct_phantom(2, (96, 96, 72))
    cam = P.orbit_camera((96, 96, 72), 160, 120, 0.6, 0.35, 40.0)
    r = Renderer(0)
    try:
        r.upload_volume(vol, 4095.0)
        r.set_camera(cam)
        outs = []
        for skip in (False, True):
            p = vr.make_surface_params(step=2.0, iso_lo=2200.0, iso_hi=4095.0, refine=6,
                                       grad="zucker_hummel", skip_empty=skip)
            img, depth = r.render_surface(params=p)
            outs.append((img.clone(), depth.clone()))
        torch.cuda.synchronize()
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
        assert torch.isfinite(outs[1][1]).sum().item() > 100
    finally:
        r.close()


def test_surface_edge_cases_and_host_outputs():
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    vol = P.ellipsoids(33, (30, 26, 20), value_max=255.0, dtype=np.uint8)
    cam = P.orbit_camera((30, 26, 20), 33, 17, 0.9, 0.2, 40.0)
    # a window above every value: no hit anywhere
    g_img, g_depth = _gpu_surface(vol, 255.0, cam, iso_lo=300.0, iso_hi=400.0)
    assert np.all(g_img == 0.0) and np.all(np.isinf(g_depth))
    # a window holding every value: every ray that meets the box hits at its entry point
    g_img, g_depth = _gpu_surface(vol, 255.0, cam, iso_lo=-1.0, iso_hi=1000.0)
    o_img, o_depth = _oracle_surface(vol, 255.0, cam, iso_lo=-1.0, iso_hi=1000.0)
    assert np.array_equal(g_depth, o_depth)
    # single-voxel and single-slice volumes
    for tiny in (np.full((1, 1, 1), 200, np.uint8), P.ellipsoids(34, (9, 7, 1), value_max=255.0,
                                                                  dtype=np.uint8)):
        nz, ny, nx = tiny.shape
        c = P.camera([nx / 2 + 5.0, ny / 2 - 7.0, nz / 2 + 9.0], [nx / 2, ny / 2, nz / 2],
                     [0, 0, 1], 16, 12, fov_y_deg=60.0)
        g_img, g_depth = _gpu_surface(tiny, 255.0, c, step=0.25, iso_lo=100.0, iso_hi=255.0)
        o_img, o_depth = _oracle_surface(tiny, 255.0, c, step=0.25, iso_lo=100.0, iso_hi=255.0)
        assert np.array_equal(g_depth, o_depth)
        assert_image_parity(g_img, o_img, f"tiny {tiny.shape}")
    # host outputs equal device outputs
    r = Renderer(0)
    try:
        r.upload_volume(vol, 255.0)
        r.set_camera(cam)
        p = vr.make_surface_params(step=1.0, iso_lo=90.0, refine=4)
        d_img, d_depth = r.render_surface(params=p)
        h_img = np.full((17, 33, 4), np.nan, np.float32)
        h_depth = np.full((17, 33), np.nan, np.float32)
        vr.vr_render_surface(r.ctx, p, h_img, h_depth)
        torch.cuda.synchronize()
        assert np.array_equal(h_img, d_img.cpu().numpy())
        assert np.array_equal(h_depth, d_depth.cpu().numpy())
        # invalid arguments are rejected before any work
        for bad in (dict(step=0.0), dict(iso_lo=5.0, iso_hi=4.0), dict(refine=25),
                    dict(iso_lo=float("nan")), dict(grad=7)):
            kw = dict(step=1.0, iso_lo=90.0, refine=4)
            kw.update(bad)
            with pytest.raises(vr.VrError) as e:
                vr.vr_render_surface(r.ctx, vr.make_surface_params(**kw), d_img)
            assert e.value.status == 1
        with pytest.raises(vr.VrError) as e:
            vr.vr_render_surface(r.ctx, p, None)
        assert e.value.status == 1
    finally:
        r.close()
    r = Renderer(0)
    try:
        r.upload_volume(vol, 255.0)
        with pytest.raises(vr.VrError) as e:  # no camera yet
            vr.vr_render_surface(r.ctx, vr.make_surface_params(), np.zeros((2, 2, 4), np.float32))
        assert e.value.status == 6
    finally:
        r.close()


def test_surface_full_size_ct_band():
    """The 512 x 512 x 361 CT phantom at 1920 x 1080, bone window, coarse step 2 (four times
    the direct renderer's), six refinement steps, Zucker-Hummel: a band of rows vs the oracle."""
    import torch

    w = P.workload_ct()
    img, depth = _gpu_surface(w["volume"], 4095.0, w["camera"], step=2.0, iso_lo=2200.0,
                              iso_hi=4095.0, refine=6, grad="zucker_hummel", skip_empty=True)
    rows = (520, 536)
    o_img, o_depth = _oracle_surface(w["volume"], 4095.0, w["camera"], rows=rows, step=2.0,
                                     iso_lo=2200.0, iso_hi=4095.0, refine=6, grad="zucker_hummel")
    sl = slice(*rows)
    assert np.array_equal(depth[sl], o_depth[sl])
    assert np.isfinite(o_depth[sl]).sum() > 500
    assert_image_parity(img[sl], o_img[sl], "CT bone band")
    assert np.isfinite(depth).sum() > 10000  # thin bone shells of the phantom


def test_surface_screen_rectangle_culling_drops_no_hit():
    """Only the tiles of the sampling box's screen rectangle are marched; against the oracle
    (which traces every pixel) for views that put the box off centre, fill the view, surround
    the eye or clip it."""
    shp = (30, 26, 22)
    vol = P.ellipsoids(72, shp, value_max=255.0, dtype=np.uint8)
    c = P.volume_centre(shp)
    d = P.volume_diag(shp)
    W, H = 64, 48
    cams = [P.orbit_camera(shp, W, H, 2.1, -0.7, 40.0, radius_diag=0.7),
            P.orbit_camera(shp, W, H, 1.0, 0.1, 120.0, radius_diag=0.1),
            P.camera([c[0] + 1.2 * d, c[1] + 0.3 * d, c[2]], [c[0] + 0.45 * d, c[1] + 0.4 * d, c[2]],
                     [0, 0, 1], W, H, fov_y_deg=50.0),
            P.camera([c[0], c[1] - 2 * d, c[2]], c, [0, 0, 1], W, H, ortho=True, ortho_height=14.0)]
    lo = float(np.percentile(vol, 60))
    for i, cam in enumerate(cams):
        for clip in (dict(), dict(clip_lo=(4.0, 3.0, 2.0), clip_hi=(17.5, 20.0, 12.0))):
            _check(vol, 255.0, cam, f"cam{i} {clip}", min_hits=1, step=1.0, iso_lo=lo,
                   iso_hi=3.0e38, refine=4, grad="central", **clip)
