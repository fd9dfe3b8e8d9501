"""Sort-last on one GPU: the partial images of z slabs (vr_render_partial), composited front
to back along each pixel's ray, equal the whole frame of vr_render without early
termination up to rounding (Eq. 6 is associative). The exchange itself is tested on the CPU
(tests/test_sortlast.py)."""
import math

import numpy as np
import pytest

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


SHP = (61, 47, 39)  # nx, ny, nz


def _cameras():
    return {
        "perspective": P.orbit_camera(SHP, 96, 72, 2.1, -0.35, 40.0, radius_diag=1.4),
        "ortho_above": P.orbit_camera(SHP, 80, 64, 0.5, 1.1, ortho=True, ortho_height=90.0),
        # an eye within the volume's z range: the upper rows' rays rise, the lower fall
        "eye_mid_height": P.camera((-40.0, 23.0, 19.0), (30.0, 23.0, 19.0), (0.0, 0.0, 1.0),
                                   96, 72, fov_y_deg=70.0),
    }


@pytest.mark.parametrize("cam_name", ["perspective", "ortho_above", "eye_mid_height"])
@pytest.mark.parametrize("world", [2, 3, 5])
def test_slabs_composite_to_the_whole_frame(R, cam_name, world):
    import torch
    from paper_1609_01317_gb300 import sortlast as SL, vr

    vol = P.ellipsoids(31, SHP, count=6)
    R.upload_volume(vol, 4095.0)
    R.set_transfer_function(P.tf_two_plateau(256))
    cam = _cameras()[cam_name]
    R.set_camera(cam)
    params = vr.make_params(grad="zucker_hummel", skip_empty=True, ert_threshold=2.0)
    full = R.render(params=params).clone()
    part = SL.SlabPartition(SHP[2], world)
    parts = [part.render_local(r, lambda a, b, dst: R.render_partial(a, b, params=params, out=dst),
                               torch.empty_like(full)) for r in range(world)]
    frame = SL.composite(parts, SL.ray_dz_sign(cam))
    torch.cuda.synchronize()
    err = (frame - full).abs().max().item()
    assert err <= 2e-5, err
    assert full[..., 3].max().item() > 0.5  # the frame holds opaque structure
    if cam_name == "eye_mid_height":
        s = SL.ray_dz_sign(cam)
        assert (s > 0).any() and (s < 0).any()


def test_whole_range_is_the_frame_and_bad_windows_are_refused(R):
    import torch
    from paper_1609_01317_gb300 import vr

    vol = P.ellipsoids(31, SHP, count=6)
    R.upload_volume(vol, 4095.0)
    R.set_transfer_function(P.tf_two_plateau(256))
    R.set_camera(_cameras()["perspective"])
    params = vr.make_params(grad="sobel3d", ert_threshold=2.0)
    full = R.render(params=params).clone()
    whole = R.render_partial(-math.inf, math.inf, params=params)
    torch.cuda.synchronize()
    assert torch.equal(whole, full)  # the same samples, in the same order
    host = np.full(tuple(full.shape), np.nan, np.float32)
    vr.vr_render_partial(R.ctx, params, -math.inf, math.inf, host)
    torch.cuda.synchronize()
    assert np.array_equal(host, full.cpu().numpy())
    for z0, z1 in [(5.0, 5.0), (9.0, 2.0), (float("nan"), 3.0)]:
        with pytest.raises(vr.VrError):
            R.render_partial(z0, z1, params=params)
    with pytest.raises(vr.VrError):
        R.render_partial(0.0, 8.0, params=vr.make_params(adapt_range=(400.0, 150.0)))
