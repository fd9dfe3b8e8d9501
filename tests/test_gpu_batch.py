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
