"""Pins of the oracle's first-hit surface renderer (§3.11 threshold window, §5.1 hitpoint
refinement) against closed forms and an independent brute force.

On a field that is linear in x, trilinear interpolation is exact, so the surface of a
threshold window is a plane and every ray's exact crossing distance is known in closed form;
bisection with R steps must land within step / 2^(R+1) of it (plus FP32 rounding of the
positions).  The inside test runs in FP32; the pins choose fields and cameras whose values
stay far from the window bounds except where a tie is tested on purpose.
"""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
import phantoms as P

NX, NY, NZ = 64, 40, 48


def linear_x(a, b, nx=NX, ny=NY, nz=NZ):
    """uint16 volume v = a + b x (constant in y and z), shape (nz, ny, nx)."""
    x = np.arange(nx, dtype=np.int64)
    v = a + b * x
    assert v.min() >= 0 and v.max() <= 65535
    return np.broadcast_to(v[None, None, :], (nz, ny, nx)).astype(np.uint16).copy()


def ray_of(cam, step, px, py, shape):
    hit, o, d, tn, K = oracle.ray(cam, oracle.make_params(step=step), shape, px, py)
    return np.array(o, np.float64), np.array(d, np.float64), float(tn), K, hit


def persp_cam(w=32, h=24):
    # looks along +x at the plane x = 30 from x = -40, slightly off-axis
    return P.camera([-40.0, 19.0, 23.0], [63.0, 19.5, 23.5], [0, 0, 1], w, h, fov_y_deg=30.0)


@pytest.mark.parametrize("refine", [0, 1, 3, 6, 9])
def test_hit_distance_on_a_plane_within_bisection_bound(refine):
    vol = linear_x(100, 20)  # window [700, inf) <=> x >= 30
    ov = oracle.OracleVolume(vol, 4095.0)
    step = 2.0
    cam = persp_cam()
    sp = oracle.make_surface_params(step=step, iso_lo=700.0, iso_hi=1e9, refine=refine)
    img, depth, _ = oracle.render_surface(ov, cam, sp)
    errs = []
    for py in range(cam["height"]):
        for px in range(cam["width"]):
            o, d, tn, K, hit = ray_of(cam, step, px, py, ov.shape_xyz)
            xs_exit = o[0] + (tn + K * step) * d[0]
            if not hit or K == 0 or xs_exit < 31.0:
                continue  # this ray leaves the box before the plane (or misses the box)
            t_star = (30.0 - o[0]) / d[0]
            assert np.isfinite(depth[py, px])
            errs.append(abs(depth[py, px] - t_star))
            assert img[py, px, 3] == 1.0
    assert len(errs) > 300
    bound = step / 2 ** (refine + 1)
    assert max(errs) <= bound + 1e-3
    if refine == 0:
        # without refinement the hit is the middle of the bracket: errors reach the bound
        assert max(errs) > 0.6 * bound


def test_refinement_halves_the_error():
    vol = linear_x(100, 20)
    ov = oracle.OracleVolume(vol, 4095.0)
    cam = persp_cam(48, 36)
    worst = []
    for r in range(0, 8):
        sp = oracle.make_surface_params(step=4.0, iso_lo=700.0, iso_hi=1e9, refine=r)
        _, depth, _ = oracle.render_surface(ov, cam, sp)
        e = 0.0
        for py in range(0, 36, 3):
            for px in range(0, 48, 3):
                o, d, tn, K, hit = ray_of(cam, 4.0, px, py, ov.shape_xyz)
                if hit and K and np.isfinite(depth[py, px]):
                    e = max(e, abs(depth[py, px] - (30.0 - o[0]) / d[0]))
        worst.append(e)
    for r in range(0, 6):
        assert worst[r + 1] <= 0.5 * worst[r] + 1e-4


def test_exact_threshold_counts_as_inside():
    # orthographic rays along +x enter at x = 0 (t_near = 10); with step 2 the coarse samples
    # sit at x = 1, 3, 5, ...; the window starts exactly at x = 31 (v = 720): sample k = 15 is
    # the first inside one, so without refinement the hit is the bracket middle x = 30
    vol = linear_x(100, 20)
    ov = oracle.OracleVolume(vol, 4095.0)
    cam = P.camera([-10.0, 19.5, 23.5], [0.0, 19.5, 23.5], [0, 0, 1], 8, 8, ortho=True,
                   ortho_height=8.0)
    sp = oracle.make_surface_params(step=2.0, iso_lo=720.0, iso_hi=1e9, refine=0)
    _, depth, _ = oracle.render_surface(ov, cam, sp)
    assert np.all(depth == np.float32(40.0))


def test_entry_point_inside_is_the_hit():
    vol = linear_x(100, 20)
    ov = oracle.OracleVolume(vol, 4095.0)
    # from the +x side looking -x: the ray enters at x = 63 (v = 1360), already inside
    cam = P.camera([100.0, 19.5, 23.5], [0.0, 19.5, 23.5], [0, 0, 1], 8, 8, ortho=True,
                   ortho_height=8.0)
    sp = oracle.make_surface_params(step=2.0, iso_lo=700.0, iso_hi=1e9, refine=6)
    _, depth, _ = oracle.render_surface(ov, cam, sp)
    assert np.all(depth == np.float32(37.0))  # t_near = 100 - 63


def test_miss_gives_black_transparent_and_infinite_depth():
    vol = linear_x(100, 20)
    ov = oracle.OracleVolume(vol, 4095.0)
    sp = oracle.make_surface_params(step=1.0, iso_lo=5000.0, iso_hi=6000.0, refine=6)
    img, depth, n = oracle.render_surface(ov, persp_cam(), sp)
    assert np.all(img == 0.0) and np.all(np.isinf(depth))
    assert n > 0  # coarse samples were taken


def _phong_closed_form(N, L, V, rgb, ka=0.1, kd=0.7, ks=0.2, n=20.0):
    nl = float(N @ L)
    spec = 0.0
    if nl > 0:
        R = 2 * nl * N - L
        spec = max(0.0, float(R @ V)) ** n
    return rgb * (ka + kd * max(nl, 0.0)) + ks * spec


@pytest.mark.parametrize("light", [None, (-1000.0, -1000.0, -1000.0), (1000.0, 1000.0, 1000.0),
                                   (-10.0, 60.0, -5.0)])
@pytest.mark.parametrize("case", ["rising", "falling"])
def test_plane_shading_closed_form_two_sided(case, light):
    # rising: v = 100 + 20x, window [700, inf): plane x = 30 entered from below the window
    # falling: v = 3000 - 20x on a 128-wide volume, window [700, 1000]: plane x = 100 entered
    # from above it -- the outward normal faces away and must be turned to the viewer
    if case == "rising":
        vol, lo, hi, xp = linear_x(100, 20), 700.0, 1e9, 30.0
    else:
        vol, lo, hi, xp = linear_x(3000, -20, nx=128), 700.0, 1000.0, 100.0
    ov = oracle.OracleVolume(vol, 4095.0)
    cam = P.camera([-40.0, 19.0, 23.0], [127.0, 19.5, 23.5], [0, 0, 1], 24, 16, fov_y_deg=25.0)
    rgb = np.array([0.9, 0.6, 0.3])
    # light None: the headlight; else a point light at a fixed position (§3.8: the paper's
    # (-1000, -1000, -1000) and (1000, 1000, 1000), and one near the plane), where L points
    # from the hit to the light and V from the hit to the eye
    kw = {} if light is None else {"light": light, "headlight": False}
    sp = oracle.make_surface_params(step=1.0, iso_lo=lo, iso_hi=hi, refine=8, color=tuple(rgb),
                                    grad="central", **kw)
    img, depth, _ = oracle.render_surface(ov, cam, sp)
    eye = np.array(cam["eye"], np.float64)
    lpos = eye if light is None else np.array(light, np.float64)
    lit = 0
    checked = 0
    for py in range(cam["height"]):
        for px in range(cam["width"]):
            o, d, tn, K, hit = ray_of(cam, 1.0, px, py, ov.shape_xyz)
            if not np.isfinite(depth[py, px]):
                continue
            assert abs(depth[py, px] - (xp - o[0]) / d[0]) <= 1.0 / 2 ** 9 + 1e-3
            p = o + float(depth[py, px]) * d
            N = np.array([-1.0, 0.0, 0.0])  # faces the camera, which looks along +x
            L = (lpos - p) / np.linalg.norm(lpos - p)
            V = (eye - p) / np.linalg.norm(eye - p)
            want = _phong_closed_form(N, L, V, rgb)
            np.testing.assert_allclose(img[py, px, :3], want, rtol=0, atol=1e-12)
            assert img[py, px, 3] == 1.0
            lit += float(N @ L) > 0
            checked += 1
    assert checked > 100  # rays that leave through the y / z faces first see no plane
    if light is None or light[0] < 0:
        assert lit == checked  # the lit side: diffuse (and specular) terms are exercised


def test_first_hit_index_matches_independent_trilinear_scan():
    # smooth random field; positions along each ray from the FP32 ray, values by scipy's
    # trilinear interpolation (clamp-to-edge), first coarse sample inside the window
    vol = P.blurred_random_field(11, 40)  # float32 in [0, 1], shape (40, 40, 40)
    vol = (vol * 4095.0).round().astype(np.uint16)
    ov = oracle.OracleVolume(vol, 4095.0)
    lo = float(np.percentile(vol, 80))
    cam = P.orbit_camera((40, 40, 40), 48, 48, 0.7, 0.4, 40.0)
    step = 1.5
    sp = oracle.make_surface_params(step=step, iso_lo=lo, iso_hi=1e9, refine=0)
    _, depth, _ = oracle.render_surface(ov, cam, sp)
    checked = 0
    for py in range(48):
        for px in range(48):
            o, d, tn, K, hit = ray_of(cam, step, px, py, (40, 40, 40))
            if not hit or K == 0:
                assert not np.isfinite(depth[py, px])
                continue
            t = tn + (np.arange(K) + 0.5) * step
            pts = o[None, :] + t[:, None] * d[None, :]
            vals = ndimage.map_coordinates(vol.astype(np.float64), pts[:, ::-1].T, order=1,
                                           mode="nearest")
            if np.any(np.abs(vals - lo) < 1e-2):
                continue  # a coarse sample on the bound: FP32 may decide either way
            inside = np.nonzero(vals >= lo)[0]
            if inside.size == 0:
                assert not np.isfinite(depth[py, px])
                continue
            k = int(inside[0])
            if k == 0:
                continue  # the entry point decides (tested separately)
            # without refinement the hit is the middle of [t_{k-1}, t_k]
            assert abs(depth[py, px] - (tn + k * step)) <= 1e-4 * max(1.0, tn + k * step)
            checked += 1
    assert checked > 100


@pytest.mark.parametrize("refine", [0, 3, 6])
def test_curved_surface_within_bisection_bound_of_the_exact_root(refine):
    # a ball-like field v = 2000 + 100 (R - r) (integers, clamped): the window [2000, inf)
    # is a curved surface.  For rays that cross it well inside (no grazing), the exact first
    # root of the trilinear interpolant along the ray -- found independently with scipy's
    # trilinear interpolation on a fine grid and a bracketing root finder -- lies in the
    # coarse bracket, so the hit must be within step / 2^(R+1) of it
    from scipy import optimize

    n, R = 48, 15.0
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    vol = np.clip(np.rint(2000.0 + 100.0 * (R - r)), 0, 4095).astype(np.uint16)
    ov = oracle.OracleVolume(vol, 4095.0)
    vf = vol.astype(np.float64)
    cam = P.camera([c - 70.0, c + 9.0, c - 6.0], [c, c, c], [0, 0, 1], 32, 24, fov_y_deg=24.0)
    step = 1.0
    iso = 2000.0
    sp = oracle.make_surface_params(step=step, iso_lo=iso, iso_hi=1e9, refine=refine)
    _, depth, _ = oracle.render_surface(ov, cam, sp)

    def f(t, o, d):
        p = o + t * d
        return ndimage.map_coordinates(vf, p[::-1].reshape(3, 1), order=1, mode="nearest")[0] - iso

    errs = []
    for py in range(24):
        for px in range(32):
            o, d, tn, K, hit = ray_of(cam, step, px, py, (n, n, n))
            if not hit or K == 0:
                continue
            ctr = np.array([c, c, c])
            miss = np.linalg.norm(np.cross(ctr - o, d))  # distance of the ray from the centre
            if miss > 0.7 * R:
                continue  # grazing rays may cross in and out within one step
            ts = tn + (np.arange(K) + 0.5) * step
            vals = np.array([f(t, o, d) for t in ts])
            k = int(np.nonzero(vals >= 0)[0][0])
            assert k > 0  # the entry point lies outside the ball
            t_star = optimize.brentq(f, ts[k - 1], ts[k], args=(o, d), xtol=1e-10)
            errs.append(abs(depth[py, px] - t_star))
    assert len(errs) > 150
    assert max(errs) <= step / 2 ** (refine + 1) + 1e-3
