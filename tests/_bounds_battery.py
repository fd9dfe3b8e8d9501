"""Run every renderer (the tile and slab marches, row bands, z-window partial images and the
multi-view adjoint included) over volumes and views chosen to reach the edges of their buffers, in
the library named by VR_LIBRARY (the bounds-checked build), and print one JSON line with the
out-of-range index count of every context.  Run as a child process by test_gpu_bounds.py."""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import torch  # noqa: E402

import phantoms as P  # noqa: E402
from paper_1609_01317_gb300 import Renderer, vr  # noqa: E402


def views(shp):
    c = np.array(P.volume_centre(shp))
    d = max(P.volume_diag(shp), 3.0)

    def at(r, az, el):
        return list(c + r * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)]))

    return [P.camera(at(2.0 * d, 0.4, 0.3), c, [0, 0, 1], 37, 29, fov_y_deg=40.0),
            P.camera(at(0.6 * d, 2.2, -0.8), c, [0, 0, 1], 33, 21, fov_y_deg=90.0),
            P.camera(at(0.05 * d, 1.0, 0.2), c, [0, 0, 1], 24, 18, fov_y_deg=120.0),  # eye inside
            P.camera(at(1.5 * d, 0.1, -0.05), c, [0, 0, 1], 31, 17, ortho=True,
                     ortho_height=2.0 * d),
            P.camera(list(c + np.array([0.0, 0.0, 3 * d])), c, [0, 1, 0], 16, 16, ortho=True,
                     ortho_height=0.5 * d)]                                   # along -z


def main():
    counts = {}
    shapes = [(1, 1, 1), (2, 2, 2), (9, 7, 1), (17, 9, 13), (40, 36, 30)]
    dtypes = [(np.uint8, 255.0), (np.uint16, 4095.0), (np.float16, 1.0), (np.float32, 1.0)]
    for si, shp in enumerate(shapes):
        for dtype, vmax in dtypes:
            raw = P.ellipsoids(90 + si, shp, value_max=255.0, dtype=np.float32)
            vol = (raw * (vmax / 255.0)).astype(dtype)
            r = Renderer(0)
            try:
                r.upload_volume(vol, vmax)
                r.set_transfer_function(P.tf_random(91, 48, alpha_max=0.6))
                cks = []
                for cam in views(shp):
                    r.set_camera(cam)
                    H, W = cam["height"], cam["width"]
                    for grad in ("central", "sobel3d", "zucker_hummel"):
                        for kw in (dict(skip_empty=True), dict(skip_empty=False),
                                   dict(clip_lo=(0.5, 0.25, 0.0), clip_hi=(6.5, 5.0, 3.75)),
                                   dict(adapt_range=(vmax, vmax * 0.1))):
                            r.render(params=vr.make_params(grad=grad, **kw))
                        r.render(params=vr.make_params(grad=grad, march="slabs"))
                        r.render_surface(params=vr.make_surface_params(
                            step=0.75, iso_lo=0.3 * vmax, iso_hi=3.0e38, refine=5, grad=grad))
                    r.render_rows(H // 3, H - H // 4, params=vr.make_params())
                    nz = float(shp[2])
                    for z0, z1 in ((-math.inf, 0.5 * nz), (0.5 * nz, math.inf),
                                   (nz + 4.0, math.inf), (-math.inf, -2.0), (0.25, 0.3)):
                        r.render_partial(z0, z1, params=vr.make_params(grad="zucker_hummel",
                                                                       ert_threshold=2.0))
                    p = vr.make_params(grad="sobel3d", ert_threshold=0.9)
                    nb = vr.vr_checkpoint_bytes(r.ctx, p)
                    ck = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
                    off = (-ck.data_ptr()) % 256
                    img = torch.empty((H, W, 4), device="cuda")
                    vr.vr_render_forward_train(r.ctx, p, img, ck[off:off + nb], nb)
                    gv = torch.zeros(vol.shape, dtype=torch.float32, device="cuda")
                    gt = torch.zeros((48, 4), dtype=torch.float32, device="cuda")
                    gi = torch.ones((H, W, 4), device="cuda")
                    vr.vr_render_backward(r.ctx, p, ck[off:off + nb], gi, gv, gt)
                    cks.append((cam, ck, ck[off:off + nb], gi))
                # every view's adjoint in one launch
                p = vr.make_params(grad="sobel3d", ert_threshold=0.9)
                gv = torch.zeros(vol.shape, dtype=torch.float32, device="cuda")
                gt = torch.zeros((48, 4), dtype=torch.float32, device="cuda")
                vr.vr_render_backward_views(r.ctx, p, [c[0] for c in cks], [c[2] for c in cks],
                                            [c[3] for c in cks], gv, gt)
                top = np.array(shp, np.float64) - 1.0
                corners = np.array([[(k & 1) * top[0], (k >> 1 & 1) * top[1], (k >> 2 & 1) * top[2]]
                                    for k in range(8)])
                pts = np.concatenate([corners,
                                      np.random.default_rng(93).uniform(0, 1, (492, 3)) * top])
                pos = torch.from_numpy(pts.astype(np.float32)).cuda()
                out = torch.empty((500, 12), device="cuda")
                vr.vr_probe_samples(r.ctx, vr.make_params(grad="zucker_hummel"), pos, 500, out)
                outs = [torch.empty((c["height"], c["width"], 4), device="cuda")
                        for c in views(shp)]
                vr.vr_render_batch([r.ctx], views(shp), [0] * len(outs), vr.make_params(), outs)
                torch.cuda.synchronize()
                counts[f"{shp} {dtype.__name__}"] = vr.vr_read_bounds_violations(r.ctx)
            finally:
                r.close()
    print(json.dumps(counts))


if __name__ == "__main__":
    main()
