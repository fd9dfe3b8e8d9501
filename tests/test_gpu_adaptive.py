"""Adaptive sampling (§5.2) on the GPU against the FP64 oracle's definition (reading R16):
per-brick multipliers 1 / 2 / 4 from the footprint value range, samples on each brick's
coarser grid, opacity 1 - (1 - a)^m."""
import numpy as np
import pytest

import oracle
import phantoms as P
from _util import assert_image_parity

pytestmark = pytest.mark.gpu


def mixed_volume(dtype, vmax, shape=(70, 66, 40), seed=41):
    """A smooth field (small value range per region: coarse regions) with a noisy block
    (large ranges: fine regions).  Returns the volume and bounds under which the 32^3 regions
    take all three multipliers."""
    nx, ny, nz = shape
    smooth = P.blurred_random_field(seed, max(shape))[:nz, :ny, :nx].astype(np.float64)
    lo, hi = smooth.min(), smooth.max()
    vol = (0.2 + 0.6 * (smooth - lo) / (hi - lo)) * vmax
    rng = np.random.default_rng(seed)
    blk = (slice(nz // 4, nz // 2), slice(ny // 4, 3 * ny // 4), slice(nx // 3, 2 * nx // 3))
    vol[blk] += rng.normal(0, 0.08 * vmax, vol[blk].shape)
    vol = np.clip(vol, 0, vmax)
    if dtype in (np.uint8, np.uint16):
        vol = vol.round()
    vol = vol.astype(dtype)
    nr = [(n + 31) // 32 for n in (nx, ny, nz)]
    ranges = []
    for rz in range(nr[2]):
        for ry in range(nr[1]):
            for rx in range(nr[0]):
                sl = tuple(slice(max(32 * r - 1, 0), min(32 * r + 33, n - 1) + 1)
                           for r, n in ((rz, nz), (ry, ny), (rx, nx)))
                f = vol[sl].astype(np.float64)
                ranges.append(f.max() - f.min())
    r = np.sort(ranges)
    return vol, (float(r[9]), float(r[3]))


def _render_gpu(vol, vmax, tf, cam, params):
    import torch
    from paper_1609_01317_gb300 import Renderer, build

    build.build()
    r = Renderer(0)
    try:
        r.upload_volume(vol, vmax)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        img = r.render(params=params)
        torch.cuda.synchronize()
        return img.cpu().numpy(), r.stats() if params.collect_stats else None
    finally:
        r.close()


@pytest.mark.parametrize("dtype,vmax", [(np.uint8, 255.0), (np.uint16, 4095.0),
                                        (np.float16, 1.0), (np.float32, 1.0)])
@pytest.mark.parametrize("grad", ["central", "zucker_hummel"])
def test_adaptive_parity(dtype, vmax, grad):
    from paper_1609_01317_gb300 import vr

    vol, bounds = mixed_volume(dtype, vmax)
    shape = vol.shape[::-1]
    tf = P.tf_random(51, 128, alpha_max=0.08)
    for i, cam in enumerate([P.orbit_camera(shape, 47, 35, 0.6, 0.4, 40.0),
                             P.orbit_camera(shape, 40, 30, 2.5, -0.3, 0.0, ortho=True,
                                            ortho_height=70.0)]):
        ref, counts, total = oracle.render(oracle.OracleVolume(vol, vmax), tf, cam,
                                           oracle.make_params(grad=grad, adapt_range=bounds))
        for skip in (False, True):
            p = vr.make_params(grad=grad, skip_empty=skip, adapt_range=bounds,
                               collect_stats=True)
            img, st = _render_gpu(vol, vmax, tf, cam, p)
            assert_image_parity(img, ref, f"{dtype.__name__} {grad} cam{i} skip{skip}")
            assert abs(st["samples_plain"] - total) <= max(2, 1e-4 * total)
            # coarse regions of this volume are visible: fewer samples are evaluated
            _, st_reg = _render_gpu(vol, vmax, tf, cam,
                                    vr.make_params(grad=grad, skip_empty=skip, collect_stats=True))
            assert st["samples_visited"] < st_reg["samples_visited"]
    # the multipliers really vary over this volume
    regular, _, _ = oracle.render(oracle.OracleVolume(vol, vmax), tf, cam,
                                  oracle.make_params(grad=grad))
    assert np.abs(regular - ref).max() > 1e-3


def test_adaptive_skipping_bit_identical_and_fewer_samples():
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    w = P.workload_ct(width=320, height=240, shape=(128, 128, 90))
    r = Renderer(0)
    try:
        r.upload_volume(w["volume"], 4095.0)
        r.set_transfer_function(w["tf"])
        r.set_camera(w["camera"])
        outs, stats = [], []
        for skip in (False, True):
            p = vr.make_params(grad="zucker_hummel", skip_empty=skip, adapt_range=(400.0, 150.0),
                               collect_stats=True)
            outs.append(r.render(params=p).clone())
            stats.append(r.stats())
        plain = r.render(params=vr.make_params(grad="zucker_hummel", collect_stats=True)).clone()
        st_plain = r.stats()
        torch.cuda.synchronize()
        assert torch.equal(outs[0], outs[1])
        assert stats[0]["samples_plain"] == stats[1]["samples_plain"]
        # the coarse regions of this phantom are transparent air, which skipping leaves
        # anyway: adaptive sampling evaluates no more samples than the regular march
        assert stats[1]["samples_visited"] <= st_plain["samples_visited"]
    finally:
        r.close()


def test_adaptive_is_rejected_where_unsupported():
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    vol = P.ellipsoids(53, (20, 18, 16), value_max=255.0, dtype=np.uint8)
    tf = P.tf_random(52, 32)
    cam = P.orbit_camera((20, 18, 16), 16, 12, 0.5, 0.2, 40.0)
    p = vr.make_params(adapt_range=(10.0, 2.0))
    r = Renderer(0)
    try:
        r.upload_volume(vol, 255.0)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        img = torch.empty((12, 16, 4), device="cuda")
        with pytest.raises(vr.VrError) as e:
            vr.vr_checkpoint_bytes(r.ctx, p)
        assert e.value.status == 4
        with pytest.raises(vr.VrError) as e:
            vr.vr_render_batch([r.ctx], [cam], [0], p, [img])
        assert e.value.status == 4
        vt = torch.from_numpy(vol).cuda()
        tt = torch.from_numpy(tf).cuda()
        with pytest.raises(vr.VrError) as e:
            vr.vr_render_noalloc(vt, "u8", 20, 18, 16, 255.0, tt, 32, cam, p, img)
        assert e.value.status == 4
        with pytest.raises(vr.VrError) as e:
            vr.vr_render(r.ctx, vr.make_params(adapt_range=(float("nan"), 1.0)), img)
        assert e.value.status == 1
    finally:
        r.close()
