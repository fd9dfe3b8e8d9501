"""Pins of the oracle's adaptive sampling (§5.2, reading R16).

Sample k of the regular grid is taken iff k mod m == 0, with m in {1, 2, 4} the multiplier
of the 32^3 region holding the sample (from the region footprint's value range), and a taken
sample's opacity is corrected to 1 - (1 - a)^m.  Pinned here: a homogeneous slab against the
closed form, the all-m = 1 case against the regular render, and whole pixels against an
independent composition of the rule from the (separately pinned) sample, transfer-function,
gradient and shading routines.
"""
import math

import numpy as np
import pytest

import oracle
import phantoms as P


def slab_setup(value=150, shape=(24, 20, 16)):
    nx, ny, nz = shape
    vol = np.full((nz, ny, nx), value, np.uint8)
    tf = np.zeros((256, 4), np.float32)
    tf[:, 0], tf[:, 1], tf[:, 2] = 0.8, 0.5, 0.25
    tf[:, 3] = 0.03
    cam = P.ortho_axis_camera(shape, 6, 6, "+z", ortho_height=4.0)  # rays along -z
    return vol, tf, cam


@pytest.mark.parametrize("mult,bounds", [(2, (0.0, -1.0)), (4, (-1.0, 0.0)), (4, (5.0, 0.0))])
def test_homogeneous_slab_closed_form(mult, bounds):
    vol, tf, cam = slab_setup()
    ov = oracle.OracleVolume(vol, 255.0)
    params = oracle.make_params(step=0.5, grad="central", ert_threshold=2.0,
                                adapt_range=bounds)
    img, counts, _ = oracle.render(ov, tf, cam, params)
    a = float(np.float32(0.03))  # the table holds float32 entries
    rgb = np.array([0.8, 0.5, 0.25], np.float32).astype(np.float64)
    for py in range(6):
        for px in range(6):
            hit, o, d, tn, K = oracle.ray(cam, params, ov.shape_xyz, px, py)
            assert hit and K > 0
            taken = (K + mult - 1) // mult  # k = 0, m, 2m, ... < K
            A = 1.0 - (1.0 - a) ** (mult * taken)
            np.testing.assert_allclose(img[py, px, 3], A, rtol=0, atol=1e-13)
            np.testing.assert_allclose(img[py, px, :3], 0.1 * rgb * A, rtol=0, atol=1e-13)
            assert counts[py, px] == K


def test_no_qualifying_brick_equals_regular_render():
    vol = P.ellipsoids(5, (40, 36, 30), value_max=4095.0, dtype=np.uint16, noise_sigma=40.0)
    ov = oracle.OracleVolume(vol, 4095.0)
    tf = P.tf_two_plateau(256)
    cam = P.orbit_camera((40, 36, 30), 24, 20, 0.8, 0.3, 40.0)
    plain, c0, _ = oracle.render(ov, tf, cam, oracle.make_params(grad="sobel3d"))
    # every footprint holds noise (range > 0): a bound of 0 qualifies no brick
    ada, c1, _ = oracle.render(ov, tf, cam, oracle.make_params(grad="sobel3d",
                                                               adapt_range=(0.0, 0.0)))
    assert np.array_equal(plain, ada) and np.array_equal(c0, c1)


def _footprint_ranges(vol, r=32):
    nz, ny, nx = vol.shape
    nb = [(nx + r - 1) // r, (ny + r - 1) // r, (nz + r - 1) // r]
    rng = np.zeros((nb[2], nb[1], nb[0]))
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                sl = tuple(slice(max(r * b - 1, 0), min(r * b + r + 1, n - 1) + 1)
                           for b, n in ((bz, nz), (by, ny), (bx, nx)))
                blk = vol[sl].astype(np.float64)
                rng[bz, by, bx] = blk.max() - blk.min()
    return rng, nb


def _compose(ov, tf, cam, params, step, bounds, ranges, nb, px, py, grad="central"):
    """The adaptive rule written out for one pixel from the pinned per-sample routines;
    returns (C, A, kend) or None when a sample sits on a region face."""
    hit, o, d, tn, K = oracle.ray(cam, params, ov.shape_xyz, px, py)
    if not hit or K == 0:
        return None
    mults = np.where(ranges <= bounds[1], 4, np.where(ranges <= bounds[0], 2, 1))
    o64, d64 = o.astype(np.float64), d.astype(np.float64)
    ts = float(tn) + (np.arange(K) + 0.5) * float(np.float32(step))  # the FP32 step
    pts = o64[None, :] + ts[:, None] * d64[None, :]
    frac = pts / 32.0 - np.floor(pts / 32.0)
    if np.any(np.minimum(frac, 1 - frac) < 1e-5):
        return None  # a sample on a region face: FP32 may pick either region
    eye = np.array(cam["eye"], np.float32).astype(np.float64)
    C, T, kend = np.zeros(3), 1.0, K
    for k in range(K):
        b = [min(int(math.floor(pts[k, a])) >> 5, nb[a] - 1) for a in range(3)]
        m = int(mults[b[2], b[1], b[0]])
        if k % m:
            continue
        s = oracle.sample(ov, pts[k])
        rgba, _ = oracle.tf_lookup(tf, s)
        a = 1.0 - (1.0 - rgba[3]) ** m
        if a != 0.0:
            g = oracle.gradient(ov, grad, pts[k])
            gl = np.linalg.norm(g)
            N = -g / gl if gl > 1e-6 else np.zeros(3)
            L = eye - pts[k]
            L = L / np.linalg.norm(L)
            V = -d64 if cam["ortho"] else L  # headlight: V = L for a perspective camera
            C += T * a * np.asarray(oracle.shade(N, L, V, rgba[:3]))
            T *= 1.0 - a
        if 1.0 - T >= params.ert_threshold:
            kend = k + 1
            break
    return C, 1.0 - T, kend


def test_pixels_against_independent_composition():
    # 3 x 2 x 2 regions: a smooth field (small ranges) with a noisy block and a flat block
    shape = (96, 64, 48)
    smooth = P.blurred_random_field(7, 96)[:48, :64, :96]
    vol = (40 + 150 * (smooth - smooth.min()) / (smooth.max() - smooth.min())).round()
    rng = np.random.default_rng(9)
    vol[0:24, 0:32, 0:32] += rng.integers(-40, 41, (24, 32, 32))
    vol[24:48, 32:64, 64:96] = 120
    vol = np.clip(vol, 0, 255).astype(np.uint8)
    ov = oracle.OracleVolume(vol, 255.0)
    tf = P.tf_random(12, 64, alpha_max=0.2)
    cam = P.orbit_camera(shape, 32, 24, 0.4, 0.5, 40.0)
    ranges, nb = _footprint_ranges(vol)
    r4, r2 = np.sort(ranges.ravel())[[2, 6]]  # several regions at each multiplier
    bounds = (float(r2), float(r4))
    params = oracle.make_params(step=0.7, grad="central", ert_threshold=0.99,
                                adapt_range=bounds)
    img, counts, _ = oracle.render(ov, tf, cam, params)
    mults = np.where(ranges <= bounds[1], 4, np.where(ranges <= bounds[0], 2, 1))
    assert (mults == 4).any() and (mults == 2).any() and (mults == 1).any()
    checked = 0
    for py in range(24):
        for px in range(32):
            r = _compose(ov, tf, cam, params, 0.7, bounds, ranges, nb, px, py)
            if r is None:
                continue
            C, A, kend = r
            np.testing.assert_allclose(img[py, px, :3], C, rtol=0, atol=1e-12)
            np.testing.assert_allclose(img[py, px, 3], A, rtol=0, atol=1e-12)
            assert counts[py, px] == kend
            checked += 1
    assert checked > 100


@pytest.mark.parametrize("spike,region", [(33, 0), (31, 1)])
def test_region_footprint_reaches_one_voxel_beyond_the_region(spike, region):
    # a gentle ramp along x everywhere and one spike voxel: x = 33 lies outside region 0
    # (x < 32) but inside its footprint [-1, 33]; x = 31 lies outside region 1 (x >= 32) but
    # inside its footprint [31, 65]; the region must then sample every sample
    nx, ny, nz = 80, 40, 40
    x = np.arange(nx, dtype=np.float64)
    vol = np.broadcast_to(60 + 0.2 * x, (nz, ny, nx)).copy()
    vol[20, 20, spike] = 250
    vol = vol.round().astype(np.uint8)
    ov = oracle.OracleVolume(vol, 255.0)
    tf = np.zeros((256, 4), np.float32)
    v = np.arange(256) / 255.0
    tf[:, 0], tf[:, 1], tf[:, 2] = v, 1 - v, 0.5
    tf[:, 3] = np.clip((np.arange(256) - 50) / 400.0, 0, 1)  # opacity grows along the ramp
    cam = P.camera([-30.0, 10.5, 10.5], [79.0, 10.5, 10.5], [0, 0, 1], 8, 8, ortho=True,
                   ortho_height=6.0)
    ranges, nb = _footprint_ranges(vol)
    assert ranges[0, 0, region] > 100 and ranges[0, 0, 2] < 10
    bounds = (-1.0, 30.0)
    params = oracle.make_params(step=0.5, grad="central", ert_threshold=2.0, adapt_range=bounds)
    img, _, _ = oracle.render(ov, tf, cam, params)
    for py in range(8):
        for px in range(8):
            r = _compose(ov, tf, cam, params, 0.5, bounds, ranges, nb, px, py)
            assert r is not None
            np.testing.assert_allclose(img[py, px, :3], r[0], rtol=0, atol=1e-12)
            np.testing.assert_allclose(img[py, px, 3], r[1], rtol=0, atol=1e-12)
