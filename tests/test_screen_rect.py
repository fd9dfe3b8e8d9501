"""The screen rectangle the renderers march (vr_screen_rect, host code) never leaves out a ray
that meets the sampling box: for random cameras, volumes and clip boxes every pixel whose
oracle ray set-up (the same FP32 ray set-up as the kernels, reading R3) finds samples lies
inside the rectangle.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import phantoms as P


@pytest.fixture(scope="module")
def vr():
    from paper_1609_01317_gb300 import build, vr as _vr

    build.build()
    return _vr


def _box(shape, clip_lo, clip_hi):
    lo = [max(np.float32(c), np.float32(0.0)) for c in clip_lo]
    hi = [min(np.float32(c), np.float32(n - 1)) for c, n in zip(clip_hi, shape)]
    return [float(v) for v in lo], [float(v) for v in hi]


def test_every_hitting_ray_lies_inside_the_rectangle(vr):
    rng = np.random.default_rng(31)
    W, H = 40, 30
    culled = 0
    for trial in range(250):
        shape = tuple(int(v) for v in rng.integers(1, 50, 3))
        c = np.array(P.volume_centre(shape))
        d = max(P.volume_diag(shape), 2.0)
        az, el = rng.uniform(0, 2 * math.pi), rng.uniform(-1.4, 1.4)
        r = d * rng.choice([0.05, 0.4, 0.8, 1.5, 3.0, 6.0])
        eye = c + r * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az),
                                math.sin(el)])
        target = c + rng.normal(0.0, 0.3 * d, 3)
        ortho = bool(rng.random() < 0.3)
        cam = P.camera(list(eye), list(target), [0, 0, 1] if abs(math.sin(el)) < 0.9 else [1, 0, 0],
                       W, H, ortho=ortho, fov_y_deg=float(rng.uniform(5.0, 150.0)),
                       ortho_height=float(d * rng.uniform(0.3, 3.0)))
        if rng.random() < 0.4:
            a = rng.uniform(-2, max(shape), 3)
            b = a + rng.uniform(0.0, max(shape), 3)
            clip_lo, clip_hi = list(a), list(b)
        else:
            clip_lo, clip_hi = [-1e30] * 3, [1e30] * 3
        lo, hi = _box(shape, clip_lo, clip_hi)
        x0, y0, x1, y1 = vr.vr_screen_rect(cam, lo, hi)
        assert 0 <= x0 <= x1 <= W and 0 <= y0 <= y1 <= H
        params = oracle.make_params(step=0.5, clip_lo=clip_lo, clip_hi=clip_hi)
        for py in range(H):
            for px in range(W):
                hit, _, _, _, K = oracle.ray(cam, params, shape, px, py)
                if K > 0:
                    assert x0 <= px < x1 and y0 <= py < y1, (trial, px, py, (x0, y0, x1, y1))
        culled += (x1 - x0) * (y1 - y0) < W * H
    assert culled > 60  # the rectangle is often smaller than the image


def test_degenerate_boxes_and_arguments(vr):
    cam = P.orbit_camera((20, 20, 20), 32, 24, 0.3, 0.2, 40.0)
    assert vr.vr_screen_rect(cam, (5.0, 0.0, 0.0), (3.0, 19.0, 19.0)) == (0, 0, 0, 0)  # empty
    # a box around the eye: no culling
    eye = cam["eye"]
    assert vr.vr_screen_rect(cam, [e - 1 for e in eye], [e + 1 for e in eye]) == (0, 0, 32, 24)
    # a single point in front of the camera: a few pixels
    x0, y0, x1, y1 = vr.vr_screen_rect(cam, (9.5, 9.5, 9.5), (9.5, 9.5, 9.5))
    assert 0 < x1 - x0 <= 6 and 0 < y1 - y0 <= 6
    with pytest.raises(vr.VrError) as e:
        vr.vr_screen_rect(cam, (float("nan"), 0, 0), (1, 1, 1))
    assert e.value.status == 1
    bad = dict(cam, fov_y_deg=200.0)
    with pytest.raises(vr.VrError) as e:
        vr.vr_screen_rect(bad, (0, 0, 0), (1, 1, 1))
    assert e.value.status == 1
