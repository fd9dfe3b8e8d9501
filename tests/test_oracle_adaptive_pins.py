"""Pins of the oracle's adaptive sampling (§5.2, reading R16).

Sample k of the regular grid is taken iff k mod m == 0, with m in {1, 2, 4} the multiplier
of the 8^3 brick holding the sample (from the brick footprint's value range), and a taken
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


def _footprint_ranges(vol):
    nz, ny, nx = vol.shape
    nb = [(nx + 7) // 8, (ny + 7) // 8, (nz + 7) // 8]
    rng = np.zeros((nb[2], nb[1], nb[0]))
    for bz in range(nb[2]):
        for by in range(nb[1]):
            for bx in range(nb[0]):
                sl = tuple(slice(max(8 * b - 1, 0), min(8 * b + 9, n - 1) + 1)
                           for b, n in ((bz, nz), (by, ny), (bx, nx)))
                blk = vol[sl].astype(np.float64)
                rng[bz, by, bx] = blk.max() - blk.min()
    return rng, nb


def test_pixels_against_independent_composition():
    # a volume with flat regions (coarse bricks) and a noisy ellipsoid (fine bricks)
    shape = (40, 32, 24)
    vol = P.ellipsoids(7, shape, count=3, value_max=255.0, dtype=np.uint8, noise_sigma=0.0)
    vol = vol.copy()
    rng = np.random.default_rng(9)
    vol[8:16, 8:24, 10:30] = np.clip(vol[8:16, 8:24, 10:30].astype(int)
                                     + rng.integers(-30, 31, (8, 16, 20)), 0, 255)
    ov = oracle.OracleVolume(vol, 255.0)
    tf = P.tf_random(12, 64, alpha_max=0.2)
    cam = P.orbit_camera(shape, 32, 24, 0.4, 0.5, 40.0)
    bounds = (20.0, 4.0)  # range <= 4: every 4th sample; <= 20: every 2nd
    params = oracle.make_params(step=0.7, grad="central", ert_threshold=0.99,
                                adapt_range=bounds)
    img, counts, _ = oracle.render(ov, tf, cam, params)
    ranges, nb = _footprint_ranges(vol)
    mults = np.where(ranges <= 4.0, 4, np.where(ranges <= 20.0, 2, 1))
    assert (mults == 4).any() and (mults == 2).any() and (mults == 1).any()
    checked = 0
    for py in range(24):
        for px in range(32):
            hit, o, d, tn, K = oracle.ray(cam, params, ov.shape_xyz, px, py)
            if not hit or K == 0:
                continue
            o64, d64 = o.astype(np.float64), d.astype(np.float64)
            ts = float(tn) + (np.arange(K) + 0.5) * float(np.float32(0.7))  # the FP32 step
            pts = o64[None, :] + ts[:, None] * d64[None, :]
            frac = pts / 8.0 - np.floor(pts / 8.0)
            if np.any(np.minimum(frac, 1 - frac) < 1e-4):
                continue  # a sample on a brick face: FP32 may pick either brick
            C, T, kend = np.zeros(3), 1.0, K
            for k in range(K):
                b = [min(int(math.floor(pts[k, a])) >> 3, nb[a] - 1) for a in range(3)]
                m = int(mults[b[2], b[1], b[0]])
                if k % m:
                    continue
                s = oracle.sample(ov, pts[k])
                rgba, _ = oracle.tf_lookup(tf, s)
                a = 1.0 - (1.0 - rgba[3]) ** m
                if a != 0.0:
                    g = oracle.gradient(ov, "central", pts[k])
                    gl = np.linalg.norm(g)
                    N = -g / gl if gl > 1e-6 else np.zeros(3)
                    L = np.array(cam["eye"], np.float32).astype(np.float64) - pts[k]
                    L = L / np.linalg.norm(L)
                    c = oracle.shade(N, L, L, rgba[:3])
                    C += T * a * np.asarray(c)
                    T *= 1.0 - a
                if 1.0 - T >= 0.99:
                    kend = k + 1
                    break
            np.testing.assert_allclose(img[py, px, :3], C, rtol=0, atol=1e-12)
            np.testing.assert_allclose(img[py, px, 3], 1.0 - T, rtol=0, atol=1e-12)
            assert counts[py, px] == kend
            checked += 1
    assert checked > 100
