"""The slab march (a tile's region of the volume and its gradient records staged in shared
memory) against the record march and against the FP64 oracle.

Both marches evaluate the same samples with the same arithmetic and composite them in the
same order, so their images must agree bit for bit, with the same ray and sample counts; the
oracle parity bound is the one of every other render test.
"""
import math

import numpy as np
import pytest

import oracle
import phantoms as P
from _util import assert_image_parity

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


def both(R, vol, vmax, tf, cam, dtype=None, **kw):
    """The same frame by the record march and by the slab march, with their counters."""
    import torch

    R.upload_volume(vol, vmax, dtype)
    R.set_transfer_function(tf)
    R.set_camera(cam)
    out = []
    for march in ("records", "slabs"):
        img = R.render(collect_stats=True, march=march, **kw)
        torch.cuda.synchronize()
        out.append((img.clone(), R.stats()))
    return out


def assert_same(res, name, slabs=True):
    """Bit-identical frames and counts; `slabs`: the second render really ran the slab march."""
    import torch

    (a, sa), (b, sb) = res
    assert sa["march"] == 1 and sb["march"] == (2 if slabs else 1), (name, sa["march"], sb["march"])
    assert torch.equal(a, b), f"{name}: max diff {(a - b).abs().max().item()}"
    assert sa["rays_hit"] == sb["rays_hit"], name
    assert sa["samples_plain"] == sb["samples_plain"], name


def small_ct(nx=128, ny=128, nz=90):
    return P.workload_ct(width=320, height=200, shape=(nx, ny, nz))


@pytest.mark.parametrize("skip", [True, False])
def test_sphere_ortho_central(R, skip):
    w = P.workload_sphere_64()
    res = both(R, w["volume"], 255.0, w["tf"], w["camera"], step=0.5, grad="central",
               skip_empty=skip)
    assert_same(res, f"sphere skip={skip}")


@pytest.mark.parametrize("grad", ["central", "sobel3d", "zucker_hummel"])
@pytest.mark.parametrize("dtype", ["u16", "f16", "f32"])
def test_ct_small_every_operator_and_storage(R, grad, dtype):
    w = small_ct()
    vol = w["volume"]
    vmax = P.U12_MAX
    if dtype == "f16":
        vol, vmax = (vol.astype(np.float32) / P.U12_MAX).astype(np.float16), 1.0
    elif dtype == "f32":
        vol, vmax = vol.astype(np.float32) / P.U12_MAX, 1.0
    res = both(R, vol, vmax, w["tf"], w["camera"], dtype=dtype, step=0.5, grad=grad,
               skip_empty=True)
    assert_same(res, f"ct {grad} {dtype}")


def test_ct_small_against_the_oracle(R):
    w = small_ct(96, 96, 68)
    kw = dict(step=0.5, grad="zucker_hummel")
    res = both(R, w["volume"], P.U12_MAX, w["tf"], w["camera"], skip_empty=True, **kw)
    assert_same(res, "ct96")
    img = res[1][0].cpu().numpy().astype(np.float64)
    ref, counts, total = oracle.render(oracle.OracleVolume(w["volume"], P.U12_MAX), w["tf"],
                                       w["camera"], oracle.make_params(**kw))
    assert_image_parity(img, ref, "ct96 slabs")
    assert res[1][1]["samples_plain"] == total


def test_ragged_volume_oblique_ortho_and_point_light(R):
    vol = P.random_volume(7, (37, 29, 23), np.float32, 1.0)  # nx, ny, nz
    tf = P.tf_random(3, 256, alpha_max=0.2)
    for i, (az, el) in enumerate([(0.3, 0.2), (2.2, -0.6), (4.0, 1.1), (math.pi / 4, 0.0)]):
        cam = P.orbit_camera((37, 29, 23), 96, 80, az, el, ortho=True, ortho_height=60.0)
        for light in (None, (300.0, -200.0, 90.0)):
            kw = dict(step=0.5, grad="zucker_hummel", skip_empty=True)
            if light is not None:
                kw.update(headlight=False, light=light)
            assert_same(both(R, vol, 1.0, tf, cam, **kw), f"ragged view {i} light {light}")


def test_thin_axes_and_clip_box(R):
    tf = P.tf_random(4, 256, alpha_max=0.3)
    for shape in [(20, 17, 1), (33, 9, 2), (12, 1, 30)]:  # nx, ny, nz
        vol = P.random_volume(11, shape, np.uint16, 4095.0)
        nx, ny, nz = shape
        cam = P.orbit_camera((nx, ny, nz), 64, 48, 0.7, 0.5, ortho=True,
                             ortho_height=2.0 * max(nx, ny, nz))
        assert_same(both(R, vol, 4095.0, tf, cam, step=0.5, grad="sobel3d", skip_empty=True),
                    f"thin {shape}")
    w = small_ct()
    assert_same(both(R, w["volume"], P.U12_MAX, w["tf"], w["camera"], step=0.5,
                     grad="zucker_hummel", skip_empty=True, clip_lo=(20.0, 10.0, 5.0),
                     clip_hi=(100.0, 90.0, 60.0)), "ct clip box")


def test_eye_inside_the_volume(R):
    w = small_ct()
    cam = P.camera((64.0, 60.0, 45.0), (10.0, 100.0, 30.0), (0.0, 0.0, 1.0), 160, 120,
                   fov_y_deg=50.0)
    assert_same(both(R, w["volume"], P.U12_MAX, w["tf"], cam, step=0.5, grad="zucker_hummel",
                     skip_empty=True), "eye inside")


def test_rows_of_the_slab_frame(R):
    import torch

    w = small_ct()
    R.upload_volume(w["volume"], P.U12_MAX)
    R.set_transfer_function(w["tf"])
    R.set_camera(w["camera"])
    kw = dict(step=0.5, grad="zucker_hummel", march="slabs")
    full = R.render(**kw).clone()
    for r0, r1 in [(0, 7), (7, 100), (100, 200), (37, 38)]:
        band = R.render_rows(r0, r1, **kw)
        torch.cuda.synchronize()
        assert torch.equal(band, full[r0:r1]), (r0, r1)


def test_spread_out_rays_take_the_record_march(R):
    import torch

    # a 256^3 volume on a 48 x 48 image: neighbouring rays are ~6 voxels apart, too far for
    # a tile's region to fit in shared memory; "slabs" then renders with the records
    vol = P.random_volume(5, (256, 256, 256), np.uint8, 255.0)
    tf = P.tf_c1(256)
    cam = P.orbit_camera((256, 256, 256), 48, 48, 0.4, 0.3)
    res = both(R, vol, 255.0, tf, cam, step=0.5, grad="central", skip_empty=True)
    assert_same(res, "spread out", slabs=False)
    torch.cuda.synchronize()


def test_sparse_data_and_automatic_choice(R):
    import torch

    vol = P.vessels(5, (128, 128, 128), tubes=12, shells=2)
    tf = P.tf_two_plateau(256, soft=(1900.0, 2300.0), soft_alpha=0.35, bone_alpha=0.5)
    cam = P.orbit_camera((128, 128, 128), 400, 300, 2.3, 0.45)
    res = both(R, vol, P.U12_MAX, tf, cam, step=0.5, grad="zucker_hummel", skip_empty=True)
    assert_same(res, "sparse")
    # the automatic choice is the record march (tiles, or the ray list for sparse data)
    for _ in range(3):
        img = R.render(march="auto", step=0.5, grad="zucker_hummel", collect_stats=True)
        torch.cuda.synchronize()
        assert R.stats()["march"] == 1
        assert torch.equal(img, res[0][0])


def test_march_selector_is_validated(R):
    from paper_1609_01317_gb300 import vr

    w = P.workload_sphere_64()
    R.upload_volume(w["volume"], 255.0)
    R.set_transfer_function(w["tf"])
    R.set_camera(w["camera"])
    for bad in (-1, 3):
        with pytest.raises(vr.VrError):
            R.render(params=vr.make_params(march=bad))
    # adaptive sampling runs the record march whatever is asked
    R.render(params=vr.make_params(march="slabs", adapt_range=(400.0, 150.0), collect_stats=True))
    assert R.stats()["march"] == 1
