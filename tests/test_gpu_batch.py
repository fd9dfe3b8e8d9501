"""Batched persistent rendering (vr_batch_*): one graph-captured launch over many cameras
and volumes of uneven sizes and mixed voxel types must reproduce the single renders."""
import math

import numpy as np
import pytest

import phantoms as P

pytestmark = pytest.mark.gpu


def test_batch_matches_single_renders_and_autotunes():
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    shapes = [((24, 30, 20), np.uint8, 255.0), ((40, 40, 40), np.uint16, 4095.0),
              ((33, 17, 29), np.uint8, 255.0)]
    rends = []
    for i, (shp, dt, vmax) in enumerate(shapes):
        r = Renderer(0)
        vol = P.ellipsoids(100 + i, shp, value_max=vmax, dtype=dt)
        r.upload_volume(vol, vmax)
        r.set_transfer_function(P.tf_random(200 + i, 64, alpha_max=0.3, zero_below=8))
        rends.append(r)
    cams, owner = [], []
    for i, (shp, _, _) in enumerate(shapes):
        for c in P.seeded_orbit_cameras(300 + i, shp, 5, 48 + 8 * i, 40):
            cams.append(c)
            owner.append(i)
    params = vr.make_params(grad="central", skip_empty=True)
    outs = [torch.full((c["height"], c["width"], 4), float("nan"), device="cuda") for c in cams]
    refs = []
    for c, o in zip(cams, owner):
        rends[o].set_camera(c)
        refs.append(rends[o].render(params=params).clone())
    b = vr.vr_batch_create([r.ctx for r in rends], cams, owner, params, outs)
    try:
        vr.vr_batch_run(b)
        torch.cuda.synchronize()
        for o, ref in zip(outs, refs):
            assert torch.equal(o, ref)  # same per-ray march on the same records
        for o in outs:
            o.fill_(float("nan"))
        chosen = vr.vr_batch_autotune(b)
        assert chosen[0] in (64, 128, 256) and chosen[1] * chosen[2] == 8
        vr.vr_batch_run(b)
        torch.cuda.synchronize()
        for o, ref in zip(outs, refs):
            assert torch.equal(o, ref)
        # a render with another operator recomputes the records; the batch restores its own
        rends[1].set_camera(cams[5])
        rends[1].render(params=vr.make_params(grad="sobel3d"))
        for o in outs:
            o.fill_(float("nan"))
        vr.vr_batch_run(b)
        torch.cuda.synchronize()
        for o, ref in zip(outs, refs):
            assert torch.equal(o, ref)
        # a new volume invalidates the batch
        rends[0].upload_volume(P.ellipsoids(999, shapes[0][0], value_max=255.0, dtype=np.uint8), 255.0)
        with pytest.raises(vr.VrError) as e:
            vr.vr_batch_run(b)
        assert e.value.status == 6
    finally:
        vr.vr_batch_destroy(b)
        torch.cuda.synchronize()
        for r in rends:
            r.close()


def test_one_shot_render_batch_matches_single_renders():
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    shapes = [((20, 26, 18), np.uint16, 4095.0), ((31, 22, 27), np.uint8, 255.0)]
    rends = []
    for i, (shp, dt, vmax) in enumerate(shapes):
        r = Renderer(0)
        r.upload_volume(P.ellipsoids(400 + i, shp, value_max=vmax, dtype=dt), vmax)
        r.set_transfer_function(P.tf_random(500 + i, 48, alpha_max=0.4, zero_below=6))
        rends.append(r)
    cams, owner = [], []
    for i, (shp, _, _) in enumerate(shapes):
        for c in P.seeded_orbit_cameras(600 + i, shp, 4, 37 + 5 * i, 29):
            cams.append(c)
            owner.append(i)
    try:
        for grad in ("central", "zucker_hummel"):
            params = vr.make_params(grad=grad, skip_empty=True)
            refs = []
            for c, o in zip(cams, owner):
                rends[o].set_camera(c)
                refs.append(rends[o].render(params=params).clone())
            outs = [torch.full_like(r, float("nan")) for r in refs]
            vr.vr_render_batch([r.ctx for r in rends], cams, owner, params, outs,
                               torch.cuda.current_stream().cuda_stream or None)
            torch.cuda.synchronize()
            for o, ref in zip(outs, refs):
                assert torch.equal(o, ref)
        with pytest.raises(vr.VrError) as e:
            vr.vr_render_batch([r.ctx for r in rends], cams, [0] * (len(cams) - 1) + [-1],
                               params, outs)
        assert e.value.status == 1
    finally:
        for r in rends:
            r.close()


def _sample_pixels(img, rng, n_hit=48, n_any=16):
    """Pixel coordinates of one render: n_hit pixels whose ray reached something (alpha > 0)
    and n_any anywhere, chosen with `rng` (the image stays on the device)."""
    import torch

    H, W = img.shape[0], img.shape[1]
    hit = torch.nonzero(img[..., 3] > 0).cpu().numpy()
    pick = hit[rng.choice(len(hit), size=min(n_hit, len(hit)), replace=False)] if len(hit) else \
        np.zeros((0, 2), np.int64)
    anyp = np.stack([rng.integers(0, H, n_any), rng.integers(0, W, n_any)], axis=1)
    yx = np.concatenate([pick, anyp]).astype(np.int32)
    return yx[:, 1].copy(), yx[:, 0].copy()


def test_batch_full_scale_against_the_oracle():
    """The batched workload at its benchmarked size: 8 volumes (96^3 .. 384^3, uint8 / uint16
    alternating), 64 seeded orbit cameras each at 512 x 512 (512 renders), central
    differences, skipping on, one persistent launch replayed from a CUDA graph -- with the
    default launch shape and with the autotuner's choice.  Every render is compared with
    the FP64 oracle (§3.10; rays are independent, §2.2) on 64 sampled pixels: 48 whose ray
    reaches something and 16 anywhere, at the image tolerance."""
    import torch

    import oracle
    from _util import assert_image_parity
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    wl = P.workload_batch(1.0)
    rends, cams, owner = [], [], []
    for i, w in enumerate(wl):
        r = Renderer(0)
        r.upload_volume(w["volume"], w["value_max"])
        r.set_transfer_function(w["tf"])
        rends.append(r)
        cams += w["cameras"]
        owner += [i] * len(w["cameras"])
    assert len(cams) == 512
    params = vr.make_params(grad="central", skip_empty=True)
    outs = [torch.full((c["height"], c["width"], 4), float("nan"), device="cuda") for c in cams]
    b = vr.vr_batch_create([r.ctx for r in rends], cams, owner, params, outs)
    try:
        vr.vr_batch_run(b)
        torch.cuda.synchronize()
        rng = np.random.default_rng(2024)
        picks = [_sample_pixels(o, rng) for o in outs]
        got_default = [o[torch.from_numpy(py).long().cuda(), torch.from_numpy(px).long().cuda()]
                       .cpu().numpy() for o, (px, py) in zip(outs, picks)]
        chosen = vr.vr_batch_autotune(b)
        for o in outs:
            o.fill_(float("nan"))
        vr.vr_batch_run(b)
        torch.cuda.synchronize()
        got_tuned = [o[torch.from_numpy(py).long().cuda(), torch.from_numpy(px).long().cuda()]
                     .cpu().numpy() for o, (px, py) in zip(outs, picks)]
    finally:
        vr.vr_batch_destroy(b)
        torch.cuda.synchronize()
        for r in rends:
            r.close()
    ovs = [oracle.OracleVolume(w["volume"], w["value_max"]) for w in wl]
    pr = oracle.make_params(grad="central")
    refs, hits = [], 0
    for c, o, (px, py) in zip(cams, owner, picks):
        ref, counts, _ = oracle.render_pixels(ovs[o], wl[o]["tf"], c, pr, px, py)
        refs.append(ref)
        hits += int((counts > 0).sum())
    ref_all = np.concatenate(refs)
    assert hits > 20000  # most sampled pixels see the volume
    for got, what in ((got_default, "default launch"), (got_tuned, f"autotuned {chosen}")):
        g = np.concatenate(got)
        assert np.isfinite(g).all(), what
        assert_image_parity(g[:, None, :], ref_all[:, None, :], f"batch {what}")
