"""Seeded synthetic inputs for the volume ray caster: volumes, transfer functions, cameras.

The paper renders CT scans (Stanford Bunny 512x512x360 slices of 12-bit data in 16-bit
shorts, a head, a brain and a stent; §3.2 "Laden eines Volumendatensatzes").  Those scans
are not available here, so every workload is a seeded procedural phantom with the same
shape, storage type and value range.  This module holds no rendering arithmetic: it only
draws voxel values, transfer-function tables and camera placements.  Both the CUDA path
and the CPU oracle consume what it produces; neither is imported here.

Conventions
-----------
* A volume is a numpy array of shape (nz, ny, nx) in C order, i.e. x is the fastest axis
  (voxel (x, y, z) sits at world point (x, y, z), spacing 1).
* A transfer function is a float32 array of shape (n, 4): RGBA per entry, entry i covering
  the normalised value i / (n - 1).
* A camera is a dict with keys eye, target, up (3 floats each), ortho (bool), fov_y_deg,
  ortho_height, width, height.
"""
from __future__ import annotations

import math

import numpy as np

U8_MAX = 255.0
U12_MAX = 4095.0


# --------------------------------------------------------------------------- helpers
def _grid_box(shape_zyx, lo, hi):
    """Integer index ranges [lo, hi] (inclusive, clipped) per axis, x/y/z order."""
    nz, ny, nx = shape_zyx
    n = (nx, ny, nz)
    out = []
    for a in range(3):
        a0 = max(0, int(math.floor(lo[a])))
        a1 = min(n[a] - 1, int(math.ceil(hi[a])))
        out.append((a0, a1))
    return out


def _ellipsoid_mask(shape_zyx, centre, semi, rot=None):
    """Boolean mask and its index slices for an (optionally rotated) ellipsoid.

    Returns (slices, mask) with mask covering only the bounding box of the ellipsoid.
    """
    centre = np.asarray(centre, np.float64)
    semi = np.asarray(semi, np.float64)
    if rot is None:
        rot = np.eye(3)
    # half extent of the rotated ellipsoid along each world axis
    half = np.sqrt(((rot * semi[None, :]) ** 2).sum(axis=1))
    (x0, x1), (y0, y1), (z0, z1) = _grid_box(shape_zyx, centre - half, centre + half)
    if x1 < x0 or y1 < y0 or z1 < z0:
        return None, None
    z, y, x = np.meshgrid(np.arange(z0, z1 + 1), np.arange(y0, y1 + 1),
                          np.arange(x0, x1 + 1), indexing="ij")
    d = np.stack([x - centre[0], y - centre[1], z - centre[2]], axis=-1)
    local = d @ rot  # coordinates in the ellipsoid frame (columns of rot are its axes)
    q = ((local / semi) ** 2).sum(axis=-1)
    return (slice(z0, z1 + 1), slice(y0, y1 + 1), slice(x0, x1 + 1)), q <= 1.0


def random_rotation(rng):
    """Uniformly distributed rotation matrix (QR of a Gaussian matrix, sign-fixed)."""
    a = rng.standard_normal((3, 3))
    q, r = np.linalg.qr(a)
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# --------------------------------------------------------------------------- volumes
def sphere_u8(seed: int = 0, n: int = 64, radius: float = 24.0) -> np.ndarray:
    """Solid sphere, linear radial falloff 255 -> 40, integer noise in [-8, 8] inside.

    Sphere centred at ((n-1)/2,)*3; value 255 - 215 r / radius inside (r <= radius),
    plus uniform integer noise in [-8, 8] inside only, clamped to [0, 255]; 0 outside.
    """
    rng = np.random.default_rng(seed)
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    inside = r <= radius
    v = 255.0 - 215.0 * r / radius
    noise = rng.integers(-8, 9, size=v.shape)
    v = np.where(inside, np.clip(np.rint(v) + noise, 0, 255), 0)
    return v.astype(np.uint8)


def ellipsoids(seed: int = 1, shape=(256, 256, 256), count: int = 10,
               value_max: float = U12_MAX, noise_sigma: float = 20.0,
               dtype=np.uint16) -> np.ndarray:
    """Overlapping random ellipsoids plus Gaussian noise everywhere.

    ``shape`` is (nx, ny, nz).  Each ellipsoid: centre U[0.25, 0.75] * size per axis,
    semi-axes U[0.08, 0.3] * size (size = the mean edge length), uniform random
    rotation, intensity U[0, value_max]; intensities are summed in order, clamped to
    [0, value_max]; then Gaussian noise of ``noise_sigma`` (in value units scaled from
    the 12-bit recipe) is added everywhere, rounded and clamped.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    size = np.array([nx, ny, nz], np.float64)
    ref = float(np.mean(size))
    vol = np.zeros((nz, ny, nx), np.float64)
    for _ in range(count):
        centre = rng.uniform(0.25, 0.75, 3) * size
        semi = rng.uniform(0.08, 0.3, 3) * ref
        rot = random_rotation(rng)
        inten = rng.uniform(0.0, value_max)
        sl, m = _ellipsoid_mask(vol.shape, centre, semi, rot)
        if sl is None:
            continue
        vol[sl] += np.where(m, inten, 0.0)
    vol = np.clip(vol, 0.0, value_max)
    sigma = noise_sigma * value_max / U12_MAX
    vol = vol + rng.normal(0.0, sigma, vol.shape)
    vol = np.clip(np.rint(vol), 0.0, value_max)
    return vol.astype(dtype)


def ct_phantom(seed: int = 2, shape=(512, 512, 361), noise_sigma: float = 30.0) -> np.ndarray:
    """CT-like uint16 phantom (12-bit values): body, organs, bone shells, air at 0.

    ``shape`` is (nx, ny, nz).  At the full 512x512x361 size: a body ellipsoid with
    semi-axes (230, 180, 175) at value 1000; six organ ellipsoids inside it at
    U[1000, 1200]; four bone shells 6 voxels thick at U[2500, 3500]; Gaussian noise of
    sigma 30 inside the body only; air exactly 0.  Smaller shapes scale every length by
    the ratio to the full size (noise and values unchanged).
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    scale = np.array([nx / 512.0, ny / 512.0, nz / 361.0])
    lin = float(np.min(scale))
    centre = (np.array([nx, ny, nz], np.float64) - 1.0) / 2.0
    body_semi = np.array([230.0, 180.0, 175.0]) * scale
    vol = np.zeros((nz, ny, nx), np.float64)
    sl, body = _ellipsoid_mask(vol.shape, centre, body_semi)
    vol[sl] = np.where(body, 1000.0, 0.0)
    body_full = np.zeros(vol.shape, bool)
    body_full[sl] = body
    # organs: random ellipsoids well inside the body
    for _ in range(6):
        c = centre + rng.uniform(-0.5, 0.5, 3) * body_semi
        semi = rng.uniform(18.0, 55.0, 3) * lin
        rot = random_rotation(rng)
        val = rng.uniform(1000.0, 1200.0)
        s2, m = _ellipsoid_mask(vol.shape, c, semi, rot)
        if s2 is None:
            continue
        m = m & body_full[s2]
        vol[s2] = np.where(m, val, vol[s2])
    # bone shells: hollow ellipsoids, 6 voxels thick (scaled)
    thick = max(6.0 * lin, 1.5)
    for _ in range(4):
        c = centre + rng.uniform(-0.35, 0.35, 3) * body_semi
        semi = rng.uniform(25.0, 70.0, 3) * lin
        rot = random_rotation(rng)
        val = rng.uniform(2500.0, 3500.0)
        s2, outer = _ellipsoid_mask(vol.shape, c, semi, rot)
        if s2 is None:
            continue
        # the inner mask has its own (smaller) box: embed it in a full-size mask
        inner_full = np.zeros(vol.shape, bool)
        s3, inner_m = _ellipsoid_mask(vol.shape, c, np.maximum(semi - thick, 0.5), rot)
        if s3 is not None:
            inner_full[s3] = inner_m
        shell = outer & ~inner_full[s2] & body_full[s2]
        vol[s2] = np.where(shell, val, vol[s2])
    noise = rng.normal(0.0, noise_sigma, vol.shape)
    vol = np.where(body_full, vol + noise, 0.0)
    vol = np.clip(np.rint(vol), 0.0, U12_MAX)
    return vol.astype(np.uint16)


def vessels(seed: int = 5, shape=(512, 512, 512), tubes: int = 40, shells: int = 3,
            noise_sigma: float = 30.0) -> np.ndarray:
    """Sparse uint16 phantom (12-bit values): a tree of thin vessel-like tubes and thin
    spherical shells in empty space (air exactly 0), for the hierarchical skipping of §5.4.

    ``shape`` is (nx, ny, nz).  Every tube starts within 0.08 of the edge lengths of one
    root point (drawn in the central fifth) and follows a smooth random walk (unit steps
    whose direction turns by a small random amount, reflected at the volume faces) of
    150-400 steps, with a radius tapering from U[2, 3.5] to 1 voxel and a value
    U[2000, 3500]; each shell is 2 voxels thick with a radius U[0.04, 0.1] of the smallest
    edge, centred within 0.2 of the edges of the root, value U[2500, 3500].  Gaussian noise
    of sigma ``noise_sigma`` inside the structures only.  At the default size under 0.5 %
    of the voxels are non-zero."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    n = np.array([nx, ny, nz], np.float64)
    vol = np.zeros((nz, ny, nx), np.float64)

    def ball(p, r, val):
        (x0, x1), (y0, y1), (z0, z1) = _grid_box(vol.shape, p - r, p + r)
        if x1 < x0 or y1 < y0 or z1 < z0:
            return
        z, y, x = np.meshgrid(np.arange(z0, z1 + 1), np.arange(y0, y1 + 1),
                              np.arange(x0, x1 + 1), indexing="ij")
        m = (x - p[0]) ** 2 + (y - p[1]) ** 2 + (z - p[2]) ** 2 <= r * r
        sub = vol[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1]
        sub[m] = np.maximum(sub[m], val)

    root = rng.uniform(0.4, 0.6, 3) * (n - 1.0)
    for _ in range(tubes):
        p = root + rng.uniform(-0.08, 0.08, 3) * n
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        steps = int(rng.integers(150, 401))
        r0 = rng.uniform(2.0, 3.5)
        val = rng.uniform(2000.0, 3500.0)
        for i in range(steps):
            ball(p, r0 + (1.0 - r0) * i / steps, val)
            d = d + rng.normal(0.0, 0.12, 3)
            d /= np.linalg.norm(d)
            p = p + d
            for a in range(3):  # reflect at the faces
                if p[a] < 2.0 or p[a] > n[a] - 3.0:
                    d[a] = -d[a]
                    p[a] = min(max(p[a], 2.0), n[a] - 3.0)
    for _ in range(shells):
        c = root + rng.uniform(-0.2, 0.2, 3) * n
        radius = rng.uniform(0.04, 0.1) * float(n.min())
        val = rng.uniform(2500.0, 3500.0)
        (x0, x1), (y0, y1), (z0, z1) = _grid_box(vol.shape, c - radius - 1, c + radius + 1)
        z, y, x = np.meshgrid(np.arange(z0, z1 + 1), np.arange(y0, y1 + 1),
                              np.arange(x0, x1 + 1), indexing="ij")
        dist = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
        m = np.abs(dist - radius) <= 1.0
        sub = vol[z0:z1 + 1, y0:y1 + 1, x0:x1 + 1]
        sub[m] = np.maximum(sub[m], val)
    inside = vol > 0
    vol[inside] += rng.normal(0.0, noise_sigma, int(inside.sum()))
    vol = np.clip(np.rint(vol), 0.0, U12_MAX)
    return vol.astype(np.uint16)


def density_phantom(seed: int = 3, n: int = 128, count: int = 5) -> np.ndarray:
    """Hidden float32 density phantom in [0, 1]: five overlapping ellipsoids."""
    rng = np.random.default_rng(seed)
    vol = np.zeros((n, n, n), np.float64)
    size = np.full(3, float(n))
    for _ in range(count):
        centre = rng.uniform(0.3, 0.7, 3) * size
        semi = rng.uniform(0.1, 0.3, 3) * n
        rot = random_rotation(rng)
        val = rng.uniform(0.3, 1.0)
        sl, m = _ellipsoid_mask(vol.shape, centre, semi, rot)
        if sl is None:
            continue
        vol[sl] = np.where(m, np.maximum(vol[sl], val), vol[sl])
    return vol.astype(np.float32)


def blurred_random_field(seed: int = 4, n: int = 128, sigma: float = 2.0) -> np.ndarray:
    """Float32 U[0, 1] field blurred by a Gaussian of ``sigma`` voxels (the learnable init)."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    v = rng.uniform(0.0, 1.0, (n, n, n))
    v = gaussian_filter(v, sigma=sigma, mode="nearest")
    return v.astype(np.float32)


def batch_volumes(seed0: int = 100):
    """Eight procedural volumes of uneven sizes, uint8 / uint16 alternating.

    Returns a list of (volume, value_max) pairs; sizes are (nx, ny, nz).
    """
    sizes = [(96, 96, 96), (128, 128, 128), (160, 200, 120), (256, 256, 256),
             (300, 300, 200), (320, 320, 320), (384, 384, 384), (384, 384, 256)]
    out = []
    for i, shp in enumerate(sizes):
        if i % 2 == 0:
            v = ellipsoids(seed0 + i, shp, value_max=U8_MAX, dtype=np.uint8)
            out.append((v, U8_MAX))
        else:
            v = ellipsoids(seed0 + i, shp, value_max=U12_MAX, dtype=np.uint16)
            out.append((v, U12_MAX))
    return out


def random_volume(seed: int, shape, dtype, value_max: float) -> np.ndarray:
    """Uniform random voxels (used for brute-force and edge-case tests)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    if np.issubdtype(np.dtype(dtype), np.integer):
        return rng.integers(0, int(value_max) + 1, size=(nz, ny, nx)).astype(dtype)
    return rng.uniform(0.0, value_max, size=(nz, ny, nx)).astype(dtype)


# ------------------------------------------------------------------ transfer functions
def tf_c1(n: int = 256) -> np.ndarray:
    """Grey ramp, alpha 0 below entry 30, rising linearly to 0.05 at entry 255."""
    i = np.arange(n, dtype=np.float64)
    m = n - 1
    rgb = i / m
    lo = 30.0 * m / 255.0
    a = np.where(i < lo, 0.0, 0.05 * (i - lo) / (m - lo))
    return np.stack([rgb, rgb, rgb, a], axis=1).astype(np.float32)


def tf_two_plateau(n: int = 256, value_max: float = U12_MAX,
                   soft=(800.0, 1600.0), soft_alpha: float = 0.02,
                   bone=(2200.0, 4095.0), bone_alpha: float = 0.6,
                   ramp: float = 64.0) -> np.ndarray:
    """Two-plateau transfer function given in raw value units.

    Alpha is ``soft_alpha`` on [soft[0], soft[1]] and ``bone_alpha`` on [bone[0], bone[1]],
    each with linear ramps ``ramp`` raw values wide outside the window, 0 elsewhere.
    Soft tissue is reddish and bone white (the colour scheme of §3.7 "Farbbestimmung").
    """
    v = np.arange(n, dtype=np.float64) * value_max / (n - 1)

    def plateau(lo, hi, a):
        up = np.clip((v - (lo - ramp)) / ramp, 0.0, 1.0)
        down = np.clip(((hi + ramp) - v) / ramp, 0.0, 1.0)
        return a * np.minimum(up, down)

    a_soft = plateau(soft[0], soft[1], soft_alpha)
    a_bone = plateau(bone[0], bone[1], bone_alpha)
    alpha = np.maximum(a_soft, a_bone)
    w = np.clip((v - soft[1]) / max(bone[0] - soft[1], 1.0), 0.0, 1.0)
    tissue = np.array([0.85, 0.35, 0.28])
    white = np.array([1.0, 0.98, 0.94])
    rgb = tissue[None, :] * (1.0 - w[:, None]) + white[None, :] * w[:, None]
    return np.concatenate([rgb, alpha[:, None]], axis=1).astype(np.float32)


def tf_random(seed: int, n: int = 256, alpha_max: float = 0.3, zero_below: int = 0) -> np.ndarray:
    """Random RGBA table (alpha in [0, alpha_max]); entries below ``zero_below`` get alpha 0."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(0.0, 1.0, (n, 4))
    t[:, 3] *= alpha_max
    t[:zero_below, 3] = 0.0
    return t.astype(np.float32)


# --------------------------------------------------------------------------- cameras
def camera(eye, target, up, width, height, ortho=False, fov_y_deg=40.0, ortho_height=1.0):
    return {"eye": [float(c) for c in eye], "target": [float(c) for c in target],
            "up": [float(c) for c in up], "ortho": bool(ortho), "fov_y_deg": float(fov_y_deg),
            "ortho_height": float(ortho_height), "width": int(width), "height": int(height)}


def volume_centre(shape_xyz):
    return [(s - 1) / 2.0 for s in shape_xyz]


def volume_diag(shape_xyz):
    return float(math.sqrt(sum((s - 1) ** 2 for s in shape_xyz)))


def ortho_axis_camera(shape_xyz, width, height, axis="+z", ortho_height=None, up=None):
    """Orthographic camera on a volume axis at twice the diagonal, looking at the centre."""
    c = volume_centre(shape_xyz)
    d = 2.0 * volume_diag(shape_xyz)
    sign = 1.0 if axis[0] == "+" else -1.0
    k = "xyz".index(axis[1])
    eye = list(c)
    eye[k] += sign * d
    if up is None:
        up = [0.0, 1.0, 0.0] if k != 1 else [0.0, 0.0, 1.0]
    if ortho_height is None:
        ortho_height = float(max(shape_xyz))
    return camera(eye, c, up, width, height, ortho=True, ortho_height=ortho_height)


def orbit_camera(shape_xyz, width, height, azimuth, elevation, fov_y_deg=40.0,
                 radius_diag=2.0, up=(0.0, 0.0, 1.0), ortho=False, ortho_height=None):
    """Camera on a sphere of radius ``radius_diag`` diagonals, looking at the centre."""
    c = volume_centre(shape_xyz)
    r = radius_diag * volume_diag(shape_xyz)
    dirv = [math.cos(elevation) * math.cos(azimuth), math.cos(elevation) * math.sin(azimuth),
            math.sin(elevation)]
    eye = [c[i] + r * dirv[i] for i in range(3)]
    if ortho_height is None:
        ortho_height = float(max(shape_xyz))
    return camera(eye, c, up, width, height, ortho=ortho, fov_y_deg=fov_y_deg,
                  ortho_height=ortho_height)


def seeded_orbit_cameras(seed: int, shape_xyz, count, width, height, fov_y_deg=40.0):
    """``count`` orbit cameras: azimuth U[0, 2 pi), elevation U[-60 deg, 60 deg]."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(count):
        az = rng.uniform(0.0, 2.0 * math.pi)
        el = rng.uniform(-math.pi / 3.0, math.pi / 3.0)
        cams.append(orbit_camera(shape_xyz, width, height, az, el, fov_y_deg))
    return cams


# ------------------------------------------------------------------- named workloads
def workload_sphere_64():
    """64^3 uint8 sphere, 256x256 orthographic view on +z, central differences."""
    vol = sphere_u8(0, 64)
    shp = (64, 64, 64)
    cam = ortho_axis_camera(shp, 256, 256, "+z", ortho_height=64.0)
    return {"name": "sphere64_u8_ortho256_cd", "volume": vol, "value_max": U8_MAX,
            "tf": tf_c1(256), "camera": cam, "grad": "central", "step": 0.5,
            "skip_empty": False}


def workload_ellipsoids_256(width=1024, height=1024, shape=(256, 256, 256)):
    """256^3 uint16 ellipsoids, perspective 1024^2 (fov 40), Sobel3D, empty-space skipping."""
    vol = ellipsoids(1, shape)
    rng = np.random.default_rng(1001)
    az = rng.uniform(0.0, 2.0 * math.pi)
    el = rng.uniform(-math.pi / 4.0, math.pi / 4.0)
    cam = orbit_camera(shape, width, height, az, el, 40.0)
    return {"name": f"ellipsoids{shape[0]}_u16_persp{width}_sobel", "volume": vol,
            "value_max": U12_MAX, "tf": tf_two_plateau(256), "camera": cam, "grad": "sobel3d",
            "step": 0.5, "skip_empty": True}


def workload_ct(width=1920, height=1080, shape=(512, 512, 361), azimuth=0.6, elevation=0.35):
    """512x512x361 uint16 CT-like phantom, perspective 1920x1080 (fov 40), Zucker-Hummel."""
    vol = ct_phantom(2, shape)
    cam = orbit_camera(shape, width, height, azimuth, elevation, 40.0)
    tf = tf_two_plateau(256, soft=(900.0, 1300.0))
    return {"name": f"ct{shape[0]}x{shape[1]}x{shape[2]}_u16_persp{width}x{height}_zh",
            "volume": vol, "value_max": U12_MAX, "tf": tf, "camera": cam,
            "grad": "zucker_hummel", "step": 0.5, "skip_empty": True}


def workload_sparse(width=3840, height=2160, shape=(512, 512, 512), azimuth=2.3,
                    elevation=0.45):
    """512^3 uint16 sparse vessel phantom (seed 5), perspective 3840x2160 (fov 40, orbit
    2x diagonal), Zucker-Hummel, step 0.5, skipping + termination; transfer function: the
    tubes and shells (alpha 0.35 above raw 1800, reddish to white), air and noise floor
    transparent."""
    vol = vessels(5, shape)
    cam = orbit_camera(shape, width, height, azimuth, elevation, 40.0)
    tf = tf_two_plateau(256, soft=(1900.0, 2300.0), soft_alpha=0.35, bone=(2300.0, 4095.0),
                        bone_alpha=0.5)
    return {"name": f"vessels{shape[0]}x{shape[1]}x{shape[2]}_u16_persp{width}x{height}_zh",
            "volume": vol, "value_max": U12_MAX, "tf": tf, "camera": cam,
            "grad": "zucker_hummel", "step": 0.5, "skip_empty": True}


def workload_batch(scale: float = 1.0, cams_per_volume: int = 64, size: int = 512):
    """Eight volumes of uneven sizes (uint8 / uint16 alternating, seeds 100..107) with
    ``cams_per_volume`` seeded orbit cameras each (seeds 200..207) at size x size.
    ``scale`` shrinks every volume edge (for quick runs).  Transfer functions: two plateaus
    at the same normalised positions for both storage types."""
    vols = []
    for i, (v, vmax) in enumerate(batch_volumes()) if scale == 1.0 else enumerate(
            _scaled_batch_volumes(scale)):
        nz, ny, nx = v.shape
        tf = tf_two_plateau(256, value_max=vmax, soft=(0.2 * vmax, 0.39 * vmax),
                            bone=(0.54 * vmax, vmax), ramp=0.016 * vmax)
        cams = seeded_orbit_cameras(200 + i, (nx, ny, nz), cams_per_volume, size, size)
        vols.append({"volume": v, "value_max": vmax, "tf": tf, "cameras": cams})
    return vols


def _scaled_batch_volumes(scale: float, seed0: int = 100):
    sizes = [(96, 96, 96), (128, 128, 128), (160, 200, 120), (256, 256, 256),
             (300, 300, 200), (320, 320, 320), (384, 384, 384), (384, 384, 256)]
    out = []
    for i, shp in enumerate(sizes):
        shp = tuple(max(8, int(round(s * scale))) for s in shp)
        vmax = U8_MAX if i % 2 == 0 else U12_MAX
        dt = np.uint8 if i % 2 == 0 else np.uint16
        out.append((ellipsoids(seed0 + i, shp, value_max=vmax, dtype=dt), vmax))
    return out


def training_views(n: int = 128, width: int = 256, height: int = 256):
    """Sixteen views of an n^3 volume: 6 axis + 2 diagonal orthographic, 8 perspective orbits."""
    shp = (n, n, n)
    views = []
    for ax in ("+x", "-x", "+y", "-y", "+z", "-z"):
        views.append(ortho_axis_camera(shp, width, height, ax, ortho_height=float(n) * 1.2))
    for az, el in ((math.pi / 4, math.atan(1 / math.sqrt(2))), (5 * math.pi / 4, -0.4)):
        views.append(orbit_camera(shp, width, height, az, el, ortho=True,
                                  ortho_height=float(n) * 1.3))
    for i in range(8):
        az = 2.0 * math.pi * (i + 0.5) / 8.0
        el = 0.5 * math.sin(1.7 * i)
        views.append(orbit_camera(shp, width, height, az, el, 40.0))
    return views
