"""The march's per-sample stages (vr_probe_samples) against the oracle's per-sample routines,
stage by stage, at every quarter-voxel position of small volumes: trilinear value (§3.4),
transfer function (§3.7), operator gradient (§3.5) and Phong (§3.8).  Each stage is fed the
GPU's own output of the previous stage, so a mismatch points at one stage."""
import numpy as np
import pytest

import oracle
import phantoms as P

pytestmark = pytest.mark.gpu


def _probe(vol, vmax, tf, cam, params, pts):
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    r = Renderer(0)
    try:
        r.upload_volume(vol, vmax)
        r.set_transfer_function(tf)
        r.set_camera(cam)
        pos = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
        out = torch.empty((len(pts), 12), dtype=torch.float32, device="cuda")
        vr.vr_probe_samples(r.ctx, params, pos, len(pts), out)
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)
    finally:
        r.close()


def _grid(shape_xyz, q=4):
    axes = [np.arange(0, (n - 1) * q + 1) / q for n in shape_xyz]
    g = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    return g


@pytest.mark.parametrize("dtype,vmax", [(np.uint8, 255.0), (np.uint16, 4095.0),
                                        (np.float16, 1.0), (np.float32, 1.0)])
@pytest.mark.parametrize("grad", ["central", "sobel3d", "zucker_hummel"])
def test_probe_stages_match_the_oracle(dtype, vmax, grad):
    from paper_1609_01317_gb300 import vr

    shp = (8, 7, 6)
    rng = np.random.default_rng(81)
    raw = rng.uniform(0, vmax, shp[::-1])
    vol = (raw.round() if dtype in (np.uint8, np.uint16) else raw).astype(dtype)
    tf = P.tf_random(82, 64, alpha_max=0.5)
    ov = oracle.OracleVolume(vol, vmax)
    pts = _grid(shp)
    for cam in (P.orbit_camera(shp, 16, 12, 0.7, 0.4, 40.0),
                P.orbit_camera(shp, 16, 12, 2.0, -0.3, 0.0, ortho=True, ortho_height=12.0)):
        p = vr.make_params(grad=grad)
        out = _probe(vol, vmax, tf, cam, p, pts)
        eye = np.array(cam["eye"], np.float32).astype(np.float64)
        fwd = np.array(cam["target"], np.float64) - np.array(cam["eye"], np.float64)
        fwd /= np.linalg.norm(fwd)
        s_o = np.array([oracle.sample(ov, q) for q in pts])
        np.testing.assert_allclose(out[:, 0], s_o, rtol=0, atol=3e-6)
        rgba_o = np.array([oracle.tf_lookup(tf, s)[0] for s in out[:, 0]])
        np.testing.assert_allclose(out[:, 1:5], rgba_o, rtol=0, atol=2e-5)
        g_o = np.array([oracle.gradient(ov, grad, q) for q in pts])
        scale = np.abs(g_o).max()
        np.testing.assert_allclose(out[:, 5:8], g_o, rtol=0, atol=2e-6 * scale)
        np.testing.assert_allclose(out[:, 11], np.linalg.norm(out[:, 5:8], axis=1), rtol=2e-6,
                                   atol=1e-9)
        checked = 0
        for k in range(0, len(pts), 7):
            g = out[k, 5:8]
            gl = np.linalg.norm(g)
            if gl < 1e-4:
                continue
            N = -g / gl
            L = eye - pts[k]
            L /= np.linalg.norm(L)
            V = -fwd if cam["ortho"] else L
            nl = N @ L
            rv = 2 * nl * (N @ V) - L @ V
            if abs(nl) < 1e-4 or abs(rv) < 1e-3:
                continue  # FP32 and FP64 may take different sides of a clamp
            c_o = oracle.shade(N, L, V, out[k, 1:4])
            np.testing.assert_allclose(out[k, 8:11], c_o, rtol=0, atol=2e-5)
            checked += 1
        assert checked > 500


def test_probe_arguments_and_state():
    import torch
    from paper_1609_01317_gb300 import Renderer, build, vr

    build.build()
    r = Renderer(0)
    try:
        p = vr.make_params()
        pos = torch.zeros((4, 3), device="cuda")
        out = torch.zeros((4, 12), device="cuda")
        with pytest.raises(vr.VrError) as e:
            vr.vr_probe_samples(r.ctx, p, pos, 4, out)  # nothing uploaded yet
        assert e.value.status == 6
        vol = P.ellipsoids(83, (9, 8, 7), value_max=255.0, dtype=np.uint8)
        r.upload_volume(vol, 255.0)
        r.set_transfer_function(P.tf_random(84, 16))
        r.set_camera(P.orbit_camera((9, 8, 7), 8, 8, 0.3, 0.2, 40.0))
        with pytest.raises(vr.VrError) as e:
            vr.vr_probe_samples(r.ctx, p, pos.cpu(), 4, out)  # host positions
        assert e.value.status == 1
        with pytest.raises(vr.VrError) as e:
            vr.vr_probe_samples(r.ctx, p, pos, -1, out)
        assert e.value.status == 1
        with pytest.raises(vr.VrError) as e:
            vr.vr_probe_samples(r.ctx, vr.make_params(adapt_range=(5.0, 1.0)), pos, 4, out)
        assert e.value.status == 4
        vr.vr_probe_samples(r.ctx, p, pos, 0, out)  # nothing to do
        vr.vr_probe_samples(r.ctx, p, pos, 4, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
    finally:
        r.close()
