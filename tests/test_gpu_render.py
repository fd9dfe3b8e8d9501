"""GPU parity of the forward ray march (vr_render) against the FP64 oracle.

Images must match within 2e-3 max abs per RGBA channel on >= 99.9% of pixels and within
2e-2 on every pixel (normalised units).  Sample counts come from the kernel's counters
and are compared with the oracle's per-ray counts.
"""
import math

import numpy as np
import pytest

import oracle
import phantoms as P
from _util import assert_image_parity, image_error

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


def gpu_render(R, vol, vmax, tf, cam, dtype=None, **kw):
    import torch

    R.upload_volume(vol, vmax, dtype)
    R.set_transfer_function(tf)
    R.set_camera(cam)
    img = R.render(collect_stats=True, **kw)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), R.stats()


def oracle_render(vol, vmax, tf, cam, **kw):
    kw = dict(kw)
    kw.pop("skip_empty", None)
    kw.pop("collect_stats", None)
    pr = oracle.make_params(**kw)
    img, counts, total = oracle.render(oracle.OracleVolume(vol, vmax), tf, cam, pr)
    return img, counts, total


def test_sphere_64_ortho_central(R):
    w = P.workload_sphere_64()
    kw = dict(step=0.5, grad="central", skip_empty=False)
    img, st = gpu_render(R, w["volume"], 255.0, w["tf"], w["camera"], **kw)
    ref, counts, total = oracle_render(w["volume"], 255.0, w["tf"], w["camera"], **kw)
    assert_image_parity(img, ref, "sphere64")
    # axis-aligned rays sit on exact binary fractions: the counts agree exactly
    assert st["rays_hit"] == 252 * 252
    assert st["samples_plain"] == total == 252 * 252 * 126
    assert st["samples_visited"] == total


@pytest.mark.parametrize("skip", [False, True])
def test_ellipsoids_perspective_sobel(R, skip):
    shp = (64, 64, 64)
    vol = P.ellipsoids(1, shp)
    tf = P.tf_two_plateau(256)
    cam = P.orbit_camera(shp, 128, 112, 0.8, 0.3, 40.0)
    kw = dict(step=0.5, grad="sobel3d", skip_empty=skip)
    img, st = gpu_render(R, vol, 4095.0, tf, cam, **kw)
    ref, counts, total = oracle_render(vol, 4095.0, tf, cam, **kw)
    assert_image_parity(img, ref, f"ellipsoids skip={skip}")
    assert abs(st["samples_plain"] - total) <= 1e-4 * total + 8
    assert st["rays_hit"] == int((counts > 0).sum()) or abs(st["rays_hit"] - (counts > 0).sum()) <= 4
    if skip:
        assert st["samples_visited"] < st["samples_plain"]


@pytest.mark.parametrize("dtype", ["u16", "f16"])
def test_ct_phantom_small_zucker_hummel(R, dtype):
    shp = (96, 96, 68)
    vol = P.ct_phantom(2, shp)
    tf = P.tf_two_plateau(256, soft=(900.0, 1300.0))
    cam = P.orbit_camera(shp, 192, 108, 0.6, 0.35, 40.0)
    kw = dict(step=0.5, grad="zucker_hummel", skip_empty=True)
    if dtype == "f16":
        vol_in = (vol.astype(np.float32) / 4095.0).astype(np.float16)
        vmax = 1.0
    else:
        vol_in, vmax = vol, 4095.0
    img, st = gpu_render(R, vol_in, vmax, tf, cam, **kw)
    ref, counts, total = oracle_render(vol_in, vmax, tf, cam, **kw)
    frac, emax = assert_image_parity(img, ref, f"ct {dtype}")
    print(f"ct {dtype}: {100 * frac:.4f}% within 2e-3, max {emax:.2e}")
    assert abs(st["samples_plain"] - total) <= 1e-4 * total + 8


@pytest.mark.parametrize("dtype", ["u8", "u16", "f16", "f32"])
@pytest.mark.parametrize("op", ["central", "sobel3d", "zucker_hummel"])
def test_dtypes_and_operators_ragged_volume(R, dtype, op):
    """Ragged (non-multiple-of-8) sizes, every storage type and operator."""
    shp = (21, 13, 17)
    vmax = {"u8": 255.0, "u16": 4095.0, "f16": 1.0, "f32": 1.0}[dtype]
    npdt = {"u8": np.uint8, "u16": np.uint16, "f16": np.float16, "f32": np.float32}[dtype]
    vol = P.ellipsoids(5, shp, count=4, value_max=vmax if dtype in ("u8", "u16") else 4095.0)
    if dtype in ("f16", "f32"):
        vol = (vol.astype(np.float64) / 4095.0).astype(npdt)
    else:
        vol = vol.astype(npdt)
    tf = P.tf_random(7, 64, alpha_max=0.25, zero_below=4)
    cam = P.orbit_camera(shp, 40, 33, 2.3, -0.5, 40.0, radius_diag=1.4)
    kw = dict(step=0.7, grad=op, skip_empty=True, ert_threshold=0.97)
    img, st = gpu_render(R, vol, vmax, tf, cam, **kw)
    ref, counts, total = oracle_render(vol, vmax, tf, cam, **kw)
    assert_image_parity(img, ref, f"{dtype}/{op}")


def test_empty_space_skipping_never_changes_the_image(R):
    shp = (80, 72, 64)
    vol = P.ellipsoids(3, shp)
    tf = P.tf_two_plateau(256)
    for i, (az, el) in enumerate([(0.1, 0.2), (1.9, -0.7), (4.0, 1.0)]):
        cam = P.orbit_camera(shp, 96, 80, az, el, 40.0, radius_diag=0.9 + 0.5 * i)
        a, sa = gpu_render(R, vol, 4095.0, tf, cam, grad="zucker_hummel", skip_empty=False)
        b, sb = gpu_render(R, vol, 4095.0, tf, cam, grad="zucker_hummel", skip_empty=True)
        assert np.array_equal(a, b)
        assert sa["samples_plain"] == sb["samples_plain"]
        assert sb["samples_visited"] <= sa["samples_visited"]


def test_edge_cases(R):
    import torch

    # all-zero volume with alpha 0 at zero: transparent black everywhere
    vol = np.zeros((9, 10, 11), np.uint8)
    tf = P.tf_c1(256)
    cam = P.orbit_camera((11, 10, 9), 17, 19, 0.3, 0.2, 40.0)
    img, st = gpu_render(R, vol, 255.0, tf, cam)
    assert np.all(img == 0.0) and st["samples_shaded"] == 0
    # camera looking away: every ray misses
    away = dict(cam)
    away["target"] = [2 * away["eye"][i] - away["target"][i] for i in range(3)]
    img, st = gpu_render(R, vol, 255.0, tf, away)
    assert np.all(img == 0.0) and st["rays_hit"] == 0
    # 1x1x1, 2x2x2 and a single slice
    for shp in ((1, 1, 1), (2, 2, 2), (7, 5, 1)):
        v = P.random_volume(9, shp, np.uint8, 255.0)
        t = P.tf_random(10, 16, alpha_max=0.5)
        ctr = P.volume_centre(shp)
        c = P.camera([ctr[0] + 3.0, ctr[1] + 2.5, ctr[2] + 4.0], ctr, [0, 1, 0], 9, 7)
        img, _ = gpu_render(R, v, 255.0, t, c, grad="sobel3d")
        ref, _, _ = oracle_render(v, 255.0, t, c, grad="sobel3d")
        assert_image_parity(img, ref, f"tiny {shp}")
    # empty clip box: black
    v = P.random_volume(11, (12, 12, 12), np.uint16, 4095.0)
    t = P.tf_random(12, 32, alpha_max=0.3)
    c = P.orbit_camera((12, 12, 12), 16, 16, 0.5, 0.5, 40.0)
    img, st = gpu_render(R, v, 4095.0, t, c, clip_lo=(6, 0, 0), clip_hi=(5, 11, 11))
    assert np.all(img == 0.0)
    # a clip box that cuts the volume open; a point light; no early termination
    kw = dict(grad="zucker_hummel", clip_lo=(2.5, 1.0, 0.0), clip_hi=(9.0, 11.0, 7.25),
              headlight=False, light=(-1000.0, -1000.0, -1000.0), ert_threshold=2.0)
    img, _ = gpu_render(R, v, 4095.0, t, c, **kw)
    ref, _, _ = oracle_render(v, 4095.0, t, c, **kw)
    assert_image_parity(img, ref, "clip + point light")
    # host output buffer (copied back on the stream)
    R.upload_volume(v, 4095.0)
    R.set_transfer_function(t)
    R.set_camera(c)
    out = torch.empty((16, 16, 4), dtype=torch.float32).pin_memory()
    from paper_1609_01317_gb300 import vr

    vr.vr_render(R.ctx, vr.make_params(), out, None)
    torch.cuda.synchronize()
    dev = R.render().cpu()
    torch.cuda.synchronize()
    assert torch.equal(out, dev)


def test_invalid_arguments_and_state(R):
    import torch
    from paper_1609_01317_gb300 import vr

    fresh = vr.vr_create(0)
    try:
        out = torch.empty((4, 4, 4), device="cuda")
        with pytest.raises(vr.VrError) as e:
            vr.vr_render(fresh, vr.make_params(), out)
        assert e.value.status == 6  # no volume / TF / camera yet
        with pytest.raises(vr.VrError):
            vr.vr_upload_volume(fresh, out, "u8", 0, 4, 4, 255.0)
        with pytest.raises(vr.VrError):
            vr.vr_upload_volume(fresh, out, "u8", 4, 4, 4, -1.0)
        with pytest.raises(vr.VrError):
            vr.vr_set_transfer_function(fresh, out, 1)
        bad = P.camera([0, 0, 0], [0, 0, 0], [0, 1, 0], 4, 4)
        with pytest.raises(vr.VrError):
            vr.vr_set_camera(fresh, bad)
        bad = P.camera([0, 0, 5], [0, 0, 0], [0, 0, 1], 4, 4)  # up parallel to view
        with pytest.raises(vr.VrError):
            vr.vr_set_camera(fresh, bad)
        bad = P.camera([0, 0, 5], [0, 0, 0], [0, 1, 0], 4, 4, fov_y_deg=180.0)
        with pytest.raises(vr.VrError):
            vr.vr_set_camera(fresh, bad)
        for p in (vr.make_params(step=0.0), vr.make_params(ert_threshold=0.0),
                  vr.make_params(grad=7), vr.make_params(shininess=-1.0)):
            with pytest.raises(vr.VrError) as e:
                vr.vr_render(fresh, p, out)
            assert e.value.status == 1
    finally:
        vr.vr_destroy(fresh)


def test_full_size_ct_sampled_pixels(R):
    """512x512x361 uint16 phantom at 1920x1080 (the benchmark's launch): sampled pixels
    against the oracle, plus the sample count of those rays."""
    import torch

    w = P.workload_ct()
    vol, tf, cam = w["volume"], w["tf"], w["camera"]
    kw = dict(step=0.5, grad="zucker_hummel", skip_empty=True)
    img, st = gpu_render(R, vol, 4095.0, tf, cam, **kw)
    hit = np.argwhere(img[..., 3] > 0)
    assert len(hit) > 50000
    rng = np.random.default_rng(5)
    pick = hit[rng.choice(len(hit), 1500, replace=False)]
    edge = rng.integers(0, [cam["height"], cam["width"]], size=(300, 2))
    pick = np.concatenate([pick, edge])
    pr = oracle.make_params(step=0.5, grad="zucker_hummel")
    ref, counts, _ = oracle.render_pixels(oracle.OracleVolume(vol, 4095.0), tf, cam, pr,
                                          pick[:, 1], pick[:, 0])
    got = img[pick[:, 0], pick[:, 1]]
    assert_image_parity(got, ref, "ct full size, sampled")
    torch.cuda.synchronize()


def test_full_size_ellipsoids_sampled_pixels(R):
    """256^3 uint16 ellipsoids at 1024 x 1024 with Sobel3D and skipping (the second
    benchmark workload): sampled pixels against the oracle."""
    w = P.workload_ellipsoids_256()
    vol, tf, cam = w["volume"], w["tf"], w["camera"]
    img, _ = gpu_render(R, vol, 4095.0, tf, cam, step=w["step"], grad=w["grad"], skip_empty=True)
    hit = np.argwhere(img[..., 3] > 0)
    assert len(hit) > 20000
    rng = np.random.default_rng(7)
    pick = np.concatenate([hit[rng.choice(len(hit), 1500, replace=False)],
                           rng.integers(0, [cam["height"], cam["width"]], size=(300, 2))])
    ref, _, _ = oracle.render_pixels(oracle.OracleVolume(vol, 4095.0), tf, cam,
                                     oracle.make_params(step=w["step"], grad=w["grad"]),
                                     pick[:, 1], pick[:, 0])
    assert_image_parity(img[pick[:, 0], pick[:, 1]], ref, "ellipsoids 256, sampled")


def test_ct_4k_f16_sampled_pixels(R):
    """The same phantom stored as FP16 (raw / 4095) at 3840 x 2160 with Sobel3D: sampled
    pixels against the oracle (2.1x the rays of the benchmark frame, 4x the tiles)."""
    w = P.workload_ct(width=3840, height=2160)
    vol = (w["volume"].astype(np.float32) / 4095.0).astype(np.float16)
    tf, cam = w["tf"], w["camera"]
    img, _ = gpu_render(R, vol, 1.0, tf, cam, step=0.5, grad="sobel3d", skip_empty=True)
    hit = np.argwhere(img[..., 3] > 0)
    assert len(hit) > 200000
    rng = np.random.default_rng(6)
    pick = np.concatenate([hit[rng.choice(len(hit), 1200, replace=False)],
                           rng.integers(0, [cam["height"], cam["width"]], size=(200, 2))])
    ref, _, _ = oracle.render_pixels(oracle.OracleVolume(vol, 1.0), tf, cam,
                                     oracle.make_params(step=0.5, grad="sobel3d"),
                                     pick[:, 1], pick[:, 0])
    assert_image_parity(img[pick[:, 0], pick[:, 1]], ref, "ct 4k f16, sampled")


def test_two_contexts_on_two_streams_overlap_and_agree():
    """Host-memory uploads and host outputs on two contexts and two streams, interleaved as a
    pipelined caller would: every frame equals the single-context device render."""
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    vol = P.ellipsoids(61, (96, 80, 72), value_max=4095.0)
    tf = P.tf_two_plateau(256)
    cam = P.orbit_camera((96, 80, 72), 160, 120, 0.8, 0.3, 40.0)
    params = vr.make_params(grad="sobel3d", skip_empty=True)
    ref_r = Renderer(0)
    rs = [Renderer(0), Renderer(0)]
    try:
        ref_r.upload_volume(vol, 4095.0)
        ref_r.set_transfer_function(tf)
        ref_r.set_camera(cam)
        ref = ref_r.render(params=params).cpu()
        host_vol = torch.from_numpy(vol.view(np.int16)).pin_memory()
        host_tf = torch.from_numpy(tf).pin_memory()
        outs = [torch.full((120, 160, 4), float("nan")).pin_memory() for _ in range(2)]
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        events = [torch.cuda.Event(), torch.cuda.Event()]
        cs = vr.make_camera(cam)
        for i in range(8):
            j = i % 2
            if i >= 2:
                events[j].synchronize()
                assert torch.equal(outs[j], ref), f"frame {i - 2}"
                outs[j].fill_(float("nan"))
            h = streams[j].cuda_stream
            vr.vr_upload_volume(rs[j].ctx, host_vol, "u16", 96, 80, 72, 4095.0, h)
            vr.vr_set_transfer_function(rs[j].ctx, host_tf, 256, h)
            vr.vr_set_camera(rs[j].ctx, cs)
            vr.vr_render(rs[j].ctx, params, outs[j], h)
            events[j].record(streams[j])
        for j in range(2):
            events[j].synchronize()
            assert torch.equal(outs[j], ref)
    finally:
        torch.cuda.synchronize()
        ref_r.close()
        for r in rs:
            r.close()


def test_allocator_failure_is_reported_and_the_context_recovers():
    """An allocator callback that returns NULL makes the call fail with
    VR_ERR_OUT_OF_MEMORY before any work; once memory is available again the same context
    renders the frame of a fresh context."""
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    budget = {"left": 1}  # vr_create's own small allocation succeeds, the next one fails
    live = {}

    def alloc(nbytes, user):
        if budget["left"] <= 0:
            return None
        budget["left"] -= 1
        p = torch.cuda.caching_allocator_alloc(int(nbytes), 0)
        live[p] = nbytes
        return p

    def free(ptr, user):
        live.pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    a, f = vr.ALLOC_FN(alloc), vr.FREE_FN(free)
    ctx = vr.vr_create(0, a, f)
    vol = P.ellipsoids(62, (40, 36, 30), value_max=4095.0)
    tf = torch.from_numpy(P.tf_two_plateau(256)).cuda()
    vd = torch.from_numpy(vol.view(np.int16)).cuda()
    cam = P.orbit_camera((40, 36, 30), 48, 40, 0.5, 0.3, 40.0)
    try:
        with pytest.raises(vr.VrError) as e:
            vr.vr_upload_volume(ctx, vd, "u16", 40, 36, 30, 4095.0)
        assert e.value.status == 2
        budget["left"] = 1_000_000
        vr.vr_upload_volume(ctx, vd, "u16", 40, 36, 30, 4095.0)
        vr.vr_set_transfer_function(ctx, tf, 256)
        vr.vr_set_camera(ctx, vr.make_camera(cam))
        img = torch.empty((40, 48, 4), device="cuda")
        p = vr.make_params(grad="sobel3d")
        vr.vr_render(ctx, p, img)
        R = Renderer(0)
        try:
            R.upload_volume(vol, 4095.0)
            R.set_transfer_function(P.tf_two_plateau(256))
            R.set_camera(cam)
            ref = R.render(params=p)
            torch.cuda.synchronize()
            assert torch.equal(img, ref)
        finally:
            R.close()
    finally:
        torch.cuda.synchronize()
        vr.vr_destroy(ctx)
    assert not live  # every buffer the context took went back through the callback


def test_screen_rectangle_culling_drops_no_ray():
    """vr_render marches only the tiles of the sampling box's screen rectangle (and the adjoint
    visits only that rectangle); a checkpointed render marches every tile with the same
    arithmetic.  For cameras that put the box anywhere -- centred, partly off screen, filling
    the view, around or inside the eye, wide and narrow fields of view, orthographic, clipped
    -- the two images are bit-identical, every ray that the FP64 oracle marches has a non-zero
    recorded end index (and every other ray 0), and the image matches the oracle's."""
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    shp = (40, 36, 30)
    vol = P.ellipsoids(71, shp, value_max=4095.0)
    c = P.volume_centre(shp)
    d = P.volume_diag(shp)
    W, H = 96, 64
    cams = [P.orbit_camera(shp, W, H, a, e, fov, radius_diag=r)
            for a, e, fov, r in ((0.3, 0.2, 40.0, 2.0), (2.1, -0.7, 40.0, 0.7), (4.0, 1.2, 90.0, 0.55),
                                 (1.0, 0.1, 120.0, 0.1), (5.5, -0.3, 5.0, 3.0))]
    cams += [P.camera([c[0] + 1.2 * d, c[1] + 0.3 * d, c[2]], [c[0] + 0.45 * d, c[1] + 0.4 * d, c[2]],
                      [0, 0, 1], W, H, fov_y_deg=50.0),                      # box off to one side
             P.camera([c[0], c[1], c[2] + 0.5 * shp[2] + 0.01], [c[0], c[1], c[2] + 100.0],
                      [0, 1, 0], W, H, fov_y_deg=150.0),                     # eye on a face, looking out
             P.camera([c[0], c[1] - 2 * d, c[2]], c, [0, 0, 1], W, H, ortho=True, ortho_height=20.0),
             P.camera([c[0] + 2 * d, c[1], c[2] + 5.0], c, [0, 0, 1], W, H, ortho=True,
                      ortho_height=300.0),
             P.camera([c[0] - 0.2 * d, c[1], c[2]], c, [0, 0, 1], W, H, ortho=True,
                      ortho_height=30.0)]                                     # ortho eye inside
    clips = [dict(), dict(clip_lo=(5.0, 3.0, 2.0), clip_hi=(17.5, 30.0, 12.0)),
             dict(clip_lo=(50.0, 0.0, 0.0), clip_hi=(60.0, 35.0, 29.0))]     # last: empty box
    R = Renderer(0)
    try:
        R.upload_volume(vol, 4095.0)
        R.set_transfer_function(P.tf_two_plateau(256))
        lit = 0
        for i, cam in enumerate(cams):
            R.set_camera(cam)
            for j, clip in enumerate(clips):
                p = vr.make_params(grad="sobel3d", **clip)
                a = torch.full((H, W, 4), float("nan"), device="cuda")
                vr.vr_render(R.ctx, p, a)
                nb = vr.vr_checkpoint_bytes(R.ctx, p)
                ck = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
                off = (-ck.data_ptr()) % 256
                b = torch.full((H, W, 4), float("nan"), device="cuda")
                vr.vr_render_forward_train(R.ctx, p, b, ck[off:off + nb], nb)
                torch.cuda.synchronize()
                assert torch.equal(a, b), f"camera {i}, clip {j}"
                kend = ck[off:off + 4 * W * H].view(torch.int32).reshape(H, W).cpu().numpy()
                ref, counts, _ = oracle.render(oracle.OracleVolume(vol, 4095.0),
                                               P.tf_two_plateau(256), cam,
                                               oracle.make_params(grad="sobel3d", **clip))
                assert np.array_equal(kend > 0, counts > 0), f"camera {i}, clip {j}"
                assert_image_parity(a.cpu().numpy(), ref, f"camera {i}, clip {j}")
                lit += int((a[..., 3] > 0).sum().item() > 0)
        assert lit >= 14  # most views see the volume
    finally:
        R.close()


def test_host_transfer_function_is_free_when_the_call_returns(R):
    """A host table is staged by the call: overwriting it right after the call (before the
    stream has run the upload queued ahead of it) does not change the frame."""
    import torch
    from paper_1609_01317_gb300 import vr

    w = P.workload_ct(width=256, height=160, shape=(96, 96, 68))
    vol = torch.from_numpy(w["volume"].view(np.int16)).cuda()
    nz, ny, nx = w["volume"].shape
    params = vr.make_params(step=0.5, grad="zucker_hummel")
    cam = vr.make_camera(w["camera"])
    out = torch.empty((160, 256, 4), device="cuda")
    s = torch.cuda.Stream()
    h = s.cuda_stream
    frames = []
    for clobber in (False, True):
        table = np.ascontiguousarray(w["tf"], np.float32).copy()
        with torch.cuda.stream(s):
            torch.cuda._sleep(2_000_000)  # keep the stream busy so the copy is still queued
            vr.vr_upload_volume(R.ctx, vol, "u16", nx, ny, nz, P.U12_MAX, h)
            vr.vr_set_transfer_function(R.ctx, table, table.shape[0], h)
            if clobber:
                table[:] = 0.5  # a different table, written before the stream reaches the copy
            vr.vr_set_camera(R.ctx, cam)
            vr.vr_render(R.ctx, params, out, h)
        s.synchronize()
        frames.append(out.clone())
    assert torch.equal(frames[0], frames[1])
    assert frames[0][..., 3].max() > 0
