"""GPU parity of the adjoint (vr_render_backward) against the FP64 oracle's reverse mode
and against central finite differences of the FP64 oracle's forward pass."""
import math

import numpy as np
import pytest

import oracle
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


def gpu_grads(R, vol, tf, cam, params, wts, value_max=1.0, dtype="f32", with_kend=False):
    """Gradient of sum(wts * image) w.r.t. raw voxels and TF, through the C ABI.  With
    `with_kend`, also each ray's end index (the leading int32 array of the checkpoints)."""
    import torch
    from paper_1609_01317_gb300 import vr

    if dtype == "f32":
        R.upload_volume(torch.from_numpy(np.ascontiguousarray(vol, np.float32)).cuda(), value_max, "f32")
    else:
        R.upload_volume(vol, value_max)
    R.set_transfer_function(torch.from_numpy(np.ascontiguousarray(tf, np.float32)).cuda())
    R.set_camera(cam)
    nb = vr.vr_checkpoint_bytes(R.ctx, params)
    ck = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    off = (-ck.data_ptr()) % 256
    ckv = ck[off:off + nb]
    H, W = cam["height"], cam["width"]
    img = torch.empty((H, W, 4), device="cuda")
    vr.vr_render_forward_train(R.ctx, params, img, ckv, nb)
    g = torch.from_numpy(np.ascontiguousarray(wts, np.float32)).cuda()
    gv = torch.zeros(vol.shape, dtype=torch.float32, device="cuda")
    gt = torch.zeros(tf.shape, dtype=torch.float32, device="cuda")
    vr.vr_render_backward(R.ctx, params, ckv, g, gv, gt)
    torch.cuda.synchronize()
    out = (img.cpu().numpy(), gv.cpu().numpy().astype(np.float64),
           gt.cpu().numpy().astype(np.float64))
    if with_kend:
        kend = ckv[:4 * H * W].view(torch.int32).reshape(H, W).cpu().numpy()
        out = out + (kend,)
    return out


# element-wise tolerance of a GPU derivative against the FP64 reverse mode (reading R17):
# |g - g64| <= REL * |g64| + FLOOR * max|g64|
REL, FLOOR = 1e-3, 1e-6


def elementwise_close(a, b, rel=REL, floor=FLOOR):
    """(all within rel * |b| + floor * max|b|, worst error in units of that bound)."""
    bound = rel * np.abs(b) + floor * np.abs(b).max()
    ratio = np.abs(a - b) / np.maximum(bound, 1e-300)
    return bool((ratio <= 1.0).all()), float(ratio.max())


@pytest.mark.parametrize("op", ["central", "sobel3d", "zucker_hummel"])
@pytest.mark.parametrize("ortho", [True, False])
def test_adjoint_matches_fp64_oracle_gradient_8cube(R, op, ortho):
    from paper_1609_01317_gb300 import vr

    rng = np.random.default_rng(81)
    n = 8
    vol = rng.uniform(0.1, 0.9, (n, n, n)).astype(np.float32)
    tf = P.tf_random(82, 16, alpha_max=0.2)
    if ortho:
        cam = P.orbit_camera((n, n, n), 14, 12, 0.8, 0.5, ortho=True, ortho_height=12.0)
    else:
        cam = P.orbit_camera((n, n, n), 14, 12, 2.2, -0.4, 40.0, radius_diag=1.3)
    wts = rng.uniform(-1, 1, (12, 14, 4))
    params = vr.make_params(grad=op, skip_empty=False, ert_threshold=2.0)
    _, gv, gt = gpu_grads(R, vol, tf, cam, params, wts)
    ref_v, ref_t = oracle.render_backward(oracle.OracleVolume(vol, 1.0), tf, cam,
                                          oracle.make_params(grad=op, ert_threshold=2.0), wts)
    okv, ev = elementwise_close(gv, ref_v)
    okt, et = elementwise_close(gt, ref_t)
    assert okv and okt, (ev, et)


def test_adjoint_with_early_termination_and_skipping_uint16(R):
    """u16 storage, Sobel, early termination on: the adjoint follows the forward's end."""
    from paper_1609_01317_gb300 import vr

    rng = np.random.default_rng(83)
    shp = (12, 10, 9)
    vol = P.ellipsoids(84, shp, count=3)
    tf = P.tf_random(85, 32, alpha_max=0.5, zero_below=6)
    cam = P.orbit_camera(shp, 16, 16, 0.4, 0.6, 40.0, radius_diag=1.2)
    wts = rng.uniform(-1, 1, (16, 16, 4))
    params = vr.make_params(grad="sobel3d", skip_empty=True, ert_threshold=0.9)
    _, gv, gt, kend = gpu_grads(R, vol, tf, cam, params, wts, value_max=4095.0, dtype="u16",
                                with_kend=True)
    ov = oracle.OracleVolume(vol, 4095.0)
    pr = oracle.make_params(grad="sobel3d", ert_threshold=0.9)
    ref_v, ref_t = oracle.render_backward(ov, tf, cam, pr, wts)
    _, counts, _ = oracle.render(ov, tf, cam, pr)
    # every ray ends at the same sample in FP32 and FP64 here, so the two differentiate the
    # same piece of the loss (reading R17 (iii)) and agree element by element
    assert np.array_equal(kend, counts)
    assert (counts > 0).sum() > 100 and (counts < 60).any()
    okv, ev = elementwise_close(gv, ref_v)
    okt, et = elementwise_close(gt, ref_t)
    assert okv and okt, (ev, et)


def _project_window(cam, p, radius):
    """Pixel window (inclusive bounds) that contains every ray passing within `radius` of p."""
    eye = np.array(cam["eye"], float)
    tgt = np.array(cam["target"], float)
    up = np.array(cam["up"], float)
    f = (tgt - eye) / np.linalg.norm(tgt - eye)
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    W, H = cam["width"], cam["height"]
    q = np.asarray(p, float) - eye
    if cam["ortho"]:
        ay = cam["ortho_height"] / 2
        ax = ay * W / H
        x, y = q @ r / ax, q @ u / ay
        rx, ry = radius / ax, radius / ay
    else:
        z = q @ f
        ay = math.tan(math.radians(cam["fov_y_deg"]) / 2)
        ax = ay * W / H
        x, y = (q @ r) / z / ax, (q @ u) / z / ay
        rx, ry = radius / (z - radius) / ax * 1.2, radius / (z - radius) / ay * 1.2
    px0 = int(math.floor(((x - rx) + 1) * W / 2)) - 2
    px1 = int(math.ceil(((x + rx) + 1) * W / 2)) + 2
    py0 = int(math.floor((1 - (y + ry)) * H / 2)) - 2
    py1 = int(math.ceil((1 - (y - ry)) * H / 2)) + 2
    return max(px0, 0), min(px1, W - 1), max(py0, 0), min(py1, H - 1)


def _fd_loss(ov, tf, cam, pr, wts, win):
    px0, px1, py0, py1 = win
    xs, ys = np.meshgrid(np.arange(px0, px1 + 1), np.arange(py0, py1 + 1))
    xs, ys = xs.ravel(), ys.ravel()
    img, _, _ = oracle.render_pixels(ov, tf, cam, pr, xs, ys)
    return float((img * wts[ys, xs]).sum())


def _central_fd(loss_at, h):
    return (loss_at(h) - loss_at(-h)) / (2 * h)


def _fd_derivative(loss_at, h=1e-3):
    """Central FD with h = 1e-3 where it is well conditioned (h and h/2 agree to 2e-4);
    elsewhere the loss is too curved at that scale (the normal of a low-contrast field
    turns quickly, and shininess 20 amplifies it) and the FP64 central FD uses h = 1e-5.
    Returns (derivative, step used)."""
    d1 = _central_fd(loss_at, h)
    d2 = _central_fd(loss_at, h / 2)
    if abs(d1 - d2) <= 2e-4 * max(abs(d1), abs(d2), 1e-30):
        return d2 + (d2 - d1) / 3.0, h  # Richardson-corrected
    return _central_fd(loss_at, 1e-5), 1e-5


def _window_weights(shape, win, rng):
    """Random image-gradient weights in [-1, 1] inside the pixel window (inclusive bounds
    px0, px1, py0, py1), zero elsewhere."""
    px0, px1, py0, py1 = win
    w = np.zeros(shape)
    w[py0:py1 + 1, px0:px1 + 1] = rng.uniform(-1, 1, (py1 - py0 + 1, px1 - px0 + 1, shape[2]))
    return w


def test_gradients_match_finite_differences_and_fp64_reverse_mode_density_128(R):
    """The differentiable workload: 128^3 float32 blurred random density, learnable
    256-entry TF, central differences, early termination at 0.99, two of its 16 views at
    256 x 256.  Reading R17: (i) every checked voxel and TF entry's GPU derivative equals the
    FP64 oracle's reverse-mode derivative element-wise, within 1e-3 relative plus 1e-6 of
    the largest; (ii) where the FP64 central difference is a reference (it agrees with the
    FP64 reverse mode to 1e-4: its stencil stays on one smooth piece of the loss), the GPU
    derivative equals the finite difference within 1e-3 relative; (iii) parameters whose
    pixel window holds a ray that ends at a different sample in FP32 and FP64 are left out
    of both, and counted."""
    from paper_1609_01317_gb300 import vr

    n = 128
    vol = P.blurred_random_field(4, n)
    tf = P.tf_c1(256)
    rng = np.random.default_rng(91)
    views = P.training_views(n, 256, 256)
    ert = 0.99
    params = vr.make_params(grad="central", skip_empty=False, ert_threshold=ert)
    pr = oracle.make_params(grad="central", ert_threshold=ert)
    ov = oracle.OracleVolume(vol.astype(np.float64), 1.0)
    arr = ov.arr.reshape(-1)
    tfd = tf.astype(np.float64).copy()
    failures, checked, fd_refs, flipped, fd_rel, an_ratio = [], 0, 0, 0, [], []

    def check_param(kind, key, g, g64, scale64, loss_at):
        nonlocal checked, fd_refs
        checked += 1
        r = abs(g - g64) / (REL * abs(g64) + FLOOR * scale64)
        an_ratio.append(r)
        if not r <= 1.0:  # a NaN derivative fails too
            failures.append(("vs FP64 reverse mode", kind, key, g, g64))
        fd, h = _fd_derivative(loss_at)
        if fd != 0.0 and abs(g64 - fd) <= 1e-4 * abs(fd):
            fd_refs += 1
            fd_rel.append(abs(g - fd) / abs(fd))
            if not fd_rel[-1] <= 1e-3:
                failures.append(("vs finite difference", kind, key, g, fd, h))

    for vi in (0, 9):
        cam = views[vi]
        wts = rng.uniform(-1, 1, (256, 256, 4))
        _, gv, _, kend = gpu_grads(R, vol, tf, cam, params, wts, with_kend=True)
        ref_v, _ = oracle.render_backward(ov, tf, cam, pr, wts)
        _, counts, _ = oracle.render(ov, tf, cam, pr)
        flips = kend != counts
        scale_v = np.abs(ref_v).max()
        # voxels: half among the largest gradients, half uniformly at random
        flat = np.abs(ref_v).ravel()
        big = np.argsort(flat)[-2000:]
        picks = np.concatenate([rng.choice(big, 24, replace=False),
                                rng.choice(flat.size, 24, replace=False)])
        for idx in picks:
            z, y, x = np.unravel_index(idx, vol.shape)
            win = _project_window(cam, (x, y, z), 4.0)
            if flips[win[2]:win[3] + 1, win[0]:win[1] + 1].any():
                flipped += 1
                continue
            x0 = arr[idx]

            def loss_at(dv, idx=idx, x0=x0, win=win):
                arr[idx] = x0 + dv
                v = _fd_loss(ov, tf, cam, pr, wts, win)
                arr[idx] = x0
                return v

            check_param("voxel", (vi, int(idx)), gv.ravel()[idx], ref_v.ravel()[idx], scale_v, loss_at)
        # TF entries: 16 x 16-pixel windows of a 64 x 64 copy of the view whose rays end at
        # the same sample in FP32 and FP64; weights inside the window only
        small = dict(cam, width=64, height=64)
        _, _, _, kend_s = gpu_grads(R, vol, tf, small, params, np.zeros((64, 64, 4)),
                                    with_kend=True)
        _, counts_s, _ = oracle.render(ov, tf, small, pr)
        wins = [(x0, x0 + 15, y0, y0 + 15) for y0 in range(0, 64, 16) for x0 in range(0, 64, 16)]
        good = [w for w in wins if (counts_s[w[2]:w[3] + 1, w[0]:w[1] + 1] > 0).mean() > 0.5]
        flipped += sum(bool((kend_s != counts_s)[w[2]:w[3] + 1, w[0]:w[1] + 1].any()) for w in good)
        good = [w for w in good if not (kend_s != counts_s)[w[2]:w[3] + 1, w[0]:w[1] + 1].any()]
        for w in good[:3]:
            wts_s = _window_weights((64, 64, 4), w, rng)
            _, _, gts = gpu_grads(R, vol, tf, small, params, wts_s)
            _, ref_t = oracle.render_backward(ov, tf, small, pr, wts_s)
            scale_t = np.abs(ref_t).max()
            cand = np.argwhere(np.abs(ref_t) > 1e-3 * scale_t)
            for (i, c) in cand[rng.choice(len(cand), min(8, len(cand)), replace=False)]:
                def loss_at(dv, i=i, c=c, w=w, wts_s=wts_s):
                    t2 = tfd.copy()
                    t2[i, c] += dv
                    return _fd_loss(ov, t2, small, pr, wts_s, w)

                check_param("tf", (vi, w, int(i), int(c)), gts[i, c], ref_t[i, c], scale_t, loss_at)
    fd_rel = np.array(fd_rel)
    print(f"R17 gradient check: {checked} parameters checked against the FP64 reverse mode "
          f"(worst {max(an_ratio):.2f} of the bound); {fd_refs} with a finite-difference "
          f"reference, worst {fd_rel.max():.2e} relative; {flipped} left out (FP32 / FP64 "
          f"termination differs in the window)")
    for f in failures:
        print("  outside:", f)
    assert checked >= 128 and flipped <= 0.1 * (checked + flipped), (checked, flipped)
    assert fd_refs >= 0.75 * checked, (fd_refs, checked)
    assert not failures, failures[:10]


def test_backward_rejects_mismatched_state(R):
    import torch
    from paper_1609_01317_gb300 import vr

    vol = P.random_volume(5, (8, 8, 8), np.float32, 1.0)
    tf = P.tf_random(6, 16)
    cam = P.orbit_camera((8, 8, 8), 8, 8, 0.1, 0.2, 40.0)
    params = vr.make_params(grad="central")
    R.upload_volume(torch.from_numpy(vol).cuda(), 1.0, "f32")
    R.set_transfer_function(tf)
    R.set_camera(cam)
    nb = vr.vr_checkpoint_bytes(R.ctx, params)
    ck = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    off = (-ck.data_ptr()) % 256
    ckv = ck[off:off + nb]
    img = torch.empty((8, 8, 4), device="cuda")
    g = torch.ones_like(img)
    gv = torch.zeros((8, 8, 8), device="cuda")
    with pytest.raises(vr.VrError) as e:  # never recorded
        vr.vr_render_backward(R.ctx, params, ckv, g, gv, None)
    assert e.value.status == 6
    vr.vr_render_forward_train(R.ctx, params, img, ckv, nb)
    with pytest.raises(vr.VrError):  # different parameters
        vr.vr_render_backward(R.ctx, vr.make_params(grad="sobel3d"), ckv, g, gv, None)
    R.set_transfer_function(tf)  # a new TF invalidates the checkpoints
    with pytest.raises(vr.VrError):
        vr.vr_render_backward(R.ctx, params, ckv, g, gv, None)
    with pytest.raises(vr.VrError):  # short buffer
        vr.vr_render_forward_train(R.ctx, params, img, ckv, nb - 4)
    torch.cuda.synchronize()


def test_autograd_multi_view_training_reduces_loss(R):
    """A few Adam steps on a 32^3 density + TF towards a hidden phantom lower the loss."""
    import torch
    from paper_1609_01317_gb300 import render_differentiable, vr

    n = 32
    target_vol = torch.from_numpy(P.density_phantom(3, n)).cuda()
    tf0 = torch.from_numpy(P.tf_c1(256)).cuda()
    views = P.training_views(n, 48, 48)[::4]
    params = vr.make_params(grad="central", skip_empty=False)
    with torch.no_grad():
        targets = [render_differentiable(R, target_vol, tf0, c, params).clone() for c in views]
    vol = torch.from_numpy(P.blurred_random_field(4, n)).cuda().requires_grad_(True)
    tf = tf0.clone().requires_grad_(True)
    opt = torch.optim.Adam([vol, tf], lr=1e-2)
    losses = []
    for _ in range(15):
        opt.zero_grad()
        loss = sum(((render_differentiable(R, vol, tf, c, params) - t) ** 2).mean()
                   for c, t in zip(views, targets)) / len(views)
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert all(math.isfinite(l) for l in losses)
    assert losses[-1] < 0.8 * losses[0], losses


def test_multi_view_backward_equals_sum_of_single_views(R):
    import torch
    from paper_1609_01317_gb300 import vr

    n = 24
    vol = torch.from_numpy(P.blurred_random_field(7, n)).cuda()
    tf = torch.from_numpy(P.tf_c1(64)).cuda()
    views = P.training_views(n, 32, 32)[::3]
    params = vr.make_params(grad="zucker_hummel", skip_empty=False)
    R.upload_volume(vol, 1.0, "f32")
    R.set_transfer_function(tf)
    cks, grads = [], []
    rng = torch.Generator(device="cuda").manual_seed(5)
    for cam in views:
        R.set_camera(cam)
        nb = vr.vr_checkpoint_bytes(R.ctx, params)
        ck = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        ckv = ck[(-ck.data_ptr()) % 256:][:nb]
        img = torch.empty((32, 32, 4), device="cuda")
        vr.vr_render_forward_train(R.ctx, params, img, ckv, nb)
        cks.append((ck, ckv))
        grads.append(torch.randn((32, 32, 4), device="cuda", generator=rng))
    gv1, gt1 = torch.zeros_like(vol), torch.zeros_like(tf)
    for cam, (_, ckv), g in zip(views, cks, grads):
        R.set_camera(cam)
        vr.vr_render_backward(R.ctx, params, ckv, g, gv1, gt1)
    gv2, gt2 = torch.zeros_like(vol), torch.zeros_like(tf)
    vr.vr_render_backward_views(R.ctx, params, views, [c[1] for c in cks], grads, gv2, gt2)
    torch.cuda.synchronize()
    assert gv1.abs().max() > 0 and gt1.abs().max() > 0
    torch.testing.assert_close(gv2, gv1, rtol=1e-4, atol=1e-5 * float(gv1.abs().max()))
    torch.testing.assert_close(gt2, gt1, rtol=1e-4, atol=1e-5 * float(gt1.abs().max()))
    # a camera that does not match the recorded checkpoints is refused
    with pytest.raises(vr.VrError):
        vr.vr_render_backward_views(R.ctx, params, views[::-1], [c[1] for c in cks], grads, gv2, gt2)


def test_adjoint_skips_only_rays_that_miss_the_box(R):
    """The adjoint visits only the tiles of the box's screen rectangle: with the box off to
    one side of a perspective view (most tiles outside it), the gradients still equal the
    FP64 reverse mode element-wise (termination off, so both differentiate the same piece)."""
    from paper_1609_01317_gb300 import vr

    rng = np.random.default_rng(87)
    shp = (14, 12, 10)
    vol = rng.uniform(0.1, 0.9, (10, 12, 14)).astype(np.float32)
    tf = P.tf_random(88, 16, alpha_max=0.2)
    c, d = P.volume_centre(shp), P.volume_diag(shp)
    cam = P.camera([c[0] + 1.6 * d, c[1] + 0.35 * d, c[2]], [c[0] + 0.3 * d, c[1] + 0.6 * d, c[2]],
                   [0, 0, 1], 40, 24, fov_y_deg=50.0)
    rect = vr.vr_screen_rect(cam, (0, 0, 0), [s - 1 for s in shp])
    assert (rect[2] - rect[0]) * (rect[3] - rect[1]) < 0.6 * 40 * 24  # most tiles culled
    wts = rng.uniform(-1, 1, (24, 40, 4))
    params = vr.make_params(grad="sobel3d", skip_empty=False, ert_threshold=2.0)
    img, gv, gt = gpu_grads(R, vol, tf, cam, params, wts)
    assert (img[..., 3] > 0).sum() > 20
    ref_v, ref_t = oracle.render_backward(oracle.OracleVolume(vol, 1.0), tf, cam,
                                          oracle.make_params(grad="sobel3d", ert_threshold=2.0), wts)
    okv, ev = elementwise_close(gv, ref_v)
    okt, et = elementwise_close(gt, ref_t)
    assert okv and okt, (ev, et)
