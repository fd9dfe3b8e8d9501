"""The sparse workload of the skipping hierarchy (§5.3, §5.4): a tree of thin vessel-like tubes
and shells in empty space.  Against the FP64 oracle at a reduced size over the whole image
and at full size (512^3, 3840 x 2160) on sampled pixels; skipping (bricks, macro bricks and
super bricks) on and off give bit-identical images and sample counts."""
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


def _render(R, w, cam, **kw):
    import torch

    R.upload_volume(w["volume"], w["value_max"])
    R.set_transfer_function(w["tf"])
    R.set_camera(cam)
    img = R.render(step=w["step"], grad=w["grad"], collect_stats=True, **kw)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), R.stats()


def test_sparse_vessels_small_whole_image_and_skipping(R):
    w = P.workload_sparse(160, 120, shape=(192, 176, 160))
    vol = w["volume"]
    assert 0 < (vol > 0).mean() < 0.05
    for az in (2.3, 0.4):
        cam = P.orbit_camera((192, 176, 160), 160, 120, az, 0.45, 40.0)
        on, st_on = _render(R, w, cam, skip_empty=True)
        off, st_off = _render(R, w, cam, skip_empty=False)
        assert np.array_equal(on, off), np.abs(on - off).max()  # skipping changes no bit
        assert st_on["samples_plain"] == st_off["samples_plain"], (st_on, st_off)
        assert st_on["samples_visited"] < 0.5 * st_off["samples_visited"], (st_on, st_off)
        ref, counts, total = oracle.render(oracle.OracleVolume(vol, w["value_max"]), w["tf"], cam,
                                           oracle.make_params(step=w["step"], grad=w["grad"]))
        assert (ref[..., 3] > 0).sum() > 500
        assert abs(st_on["samples_plain"] - total) <= 1e-4 * total, (st_on, total)
        assert_image_parity(on, ref, f"sparse small, azimuth {az}")


def test_sparse_vessels_full_size_4k_sampled_pixels(R):
    w = P.workload_sparse()
    cam = w["camera"]
    img, st = _render(R, w, cam, skip_empty=True)
    hit = np.argwhere(img[..., 3] > 0)
    assert len(hit) > 20000
    rng = np.random.default_rng(9)
    pick = np.concatenate([hit[rng.choice(len(hit), 1500, replace=False)],
                           rng.integers(0, [cam["height"], cam["width"]], size=(300, 2))])
    ref, _, _ = oracle.render_pixels(oracle.OracleVolume(w["volume"], w["value_max"]), w["tf"],
                                     cam, oracle.make_params(step=w["step"], grad=w["grad"]),
                                     pick[:, 1], pick[:, 0])
    assert_image_parity(img[pick[:, 0], pick[:, 1]], ref, "sparse 4k, sampled")
