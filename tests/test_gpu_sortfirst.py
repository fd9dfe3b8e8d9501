"""Sort-first rendering on one GPU: the rows each rank of an image-space partition renders
with vr_render_rows, stitched, equal the whole frame of vr_render bit for bit (rays are
independent, §2.2).  The collectives themselves are tested on the CPU (tests/test_sortfirst.py)."""
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


@pytest.mark.parametrize("grad,ortho", [("zucker_hummel", False), ("central", True)])
def test_stitched_rows_equal_the_whole_frame(R, grad, ortho):
    import torch
    from paper_1609_01317_gb300 import sortfirst as SF, vr

    shp = (61, 47, 39)
    vol = P.ellipsoids(31, shp, count=6)
    R.upload_volume(vol, 4095.0)
    R.set_transfer_function(P.tf_two_plateau(256))
    if ortho:
        cam = P.orbit_camera(shp, 101, 77, 0.4, 0.3, ortho=True, ortho_height=70.0)
    else:
        cam = P.orbit_camera(shp, 101, 77, 2.1, -0.35, 40.0, radius_diag=1.4)
    R.set_camera(cam)
    H, W = cam["height"], cam["width"]
    params = vr.make_params(grad=grad, skip_empty=True)
    full = R.render(params=params).clone()
    busy = vr.vr_screen_rect(cam, (0, 0, 0), [s - 1 for s in shp])
    assert 0 < busy[1] < busy[3] < H  # the partition below splits a culled frame
    parts = [SF.RowPartition.from_bands(H, W, 3, busy=(busy[1], busy[3])),
             SF.RowPartition.from_bands(H, W, 8),
             SF.RowPartition.from_stripes(H, W, 2, rows=7)]
    for part in parts:
        packed = [torch.full((part.capacity, W, 4), float("nan"), device="cuda")
                  for _ in range(part.world)]
        for rank in range(part.world):
            part.render_local(rank, lambda a, b, dst: R.render_rows(a, b, params=params, out=dst),
                              packed[rank])
        frame = part.stitch(packed, torch.full((H, W, 4), float("nan"), device="cuda"))
        torch.cuda.synchronize()
        assert torch.equal(frame, full), part.per_rank
    # a band into host memory, and the band's counters add up to the frame's
    host = np.full((20, W, 4), np.nan, np.float32)
    vr.vr_render_rows(R.ctx, params, 30, 50, host)
    torch.cuda.synchronize()
    assert np.array_equal(host, full[30:50].cpu().numpy())
    pst = vr.make_params(grad=grad, skip_empty=True, collect_stats=True)
    R.render(params=pst)
    total = vr.vr_read_stats(R.ctx)
    counters = ("rays_hit", "samples_plain", "samples_visited", "samples_shaded")
    acc = {k: 0 for k in counters}
    for a, b in SF.bands(H, 4):
        vr.vr_render_rows(R.ctx, pst, a, b, torch.empty((b - a, W, 4), device="cuda"))
        st = vr.vr_read_stats(R.ctx)
        assert st["march"] == total["march"]
        for k in counters:
            acc[k] += st[k]
    assert acc == {k: total[k] for k in counters}


def test_render_rows_rejects_bad_rows(R):
    import torch
    from paper_1609_01317_gb300 import vr

    R.upload_volume(P.ellipsoids(32, (16, 16, 16), count=3), 4095.0)
    R.set_transfer_function(P.tf_two_plateau(256))
    R.set_camera(P.orbit_camera((16, 16, 16), 20, 10, 0.3, 0.2, 40.0))
    out = torch.zeros((10, 20, 4), device="cuda")
    for a, b in ((-1, 3), (3, 3), (4, 2), (0, 11)):
        with pytest.raises(vr.VrError) as e:
            vr.vr_render_rows(R.ctx, vr.make_params(), a, b, out)
        assert e.value.status == 1
