"""The seeded synthetic inputs follow the recipes the benchmarks and parity tests are quoted
on (shapes, storage types, value ranges and structure), and are reproducible from their
seeds.  CPU only."""
import numpy as np

import phantoms as P


def test_sphere_workload():
    w = P.workload_sphere_64()
    v = w["volume"]
    assert v.shape == (64, 64, 64) and v.dtype == np.uint8
    z, y, x = np.meshgrid(*(np.arange(64),) * 3, indexing="ij")
    r = np.sqrt((x - 31.5) ** 2 + (y - 31.5) ** 2 + (z - 31.5) ** 2)
    inside = r <= 24.0
    assert np.all(v[~inside] == 0)
    expect = 255.0 - 215.0 * r / 24.0
    dev = v[inside].astype(np.float64) - np.rint(expect[inside])
    assert dev.min() >= -8 and dev.max() <= 8 and np.abs(dev).mean() > 3  # noise U[-8, 8]
    assert w["camera"]["ortho"] and (w["camera"]["width"], w["camera"]["height"]) == (256, 256)
    tf = w["tf"]
    assert tf.shape == (256, 4) and np.all(tf[:30, 3] == 0) and np.isclose(tf[255, 3], 0.05)
    assert np.array_equal(v, P.workload_sphere_64()["volume"])  # seeded


def test_two_plateau_transfer_function():
    tf = P.tf_two_plateau(4096)  # one entry per raw value
    a = tf[:, 3]
    assert np.allclose(a[800:1601], 0.02) and np.allclose(a[2200:], 0.6)
    assert np.all(a[:800 - 64] == 0) and np.all(a[1600 + 64:2200 - 64] == 0)
    assert np.all(np.diff(a[800 - 64:801]) >= 0) and np.all(np.diff(a[1600:1600 + 65]) <= 0)


def test_ct_phantom_full_size():
    w = P.workload_ct()
    v = w["volume"]
    assert v.shape == (361, 512, 512) and v.dtype == np.uint16
    assert v.max() <= 4095
    cam = w["camera"]
    assert (cam["width"], cam["height"]) == (1920, 1080) and not cam["ortho"]
    # air is exactly 0 outside the body ellipsoid (semi-axes 230, 180, 175)
    c = (np.array([512, 512, 361]) - 1) / 2.0
    zz, yy, xx = np.meshgrid(np.arange(0, 361, 8), np.arange(0, 512, 8), np.arange(0, 512, 8),
                             indexing="ij")
    q = ((xx - c[0]) / 230.0) ** 2 + ((yy - c[1]) / 180.0) ** 2 + ((zz - c[2]) / 175.0) ** 2
    sub = v[::8, ::8, ::8].astype(np.float64)
    assert np.all(sub[q > 1.05] == 0)
    body = sub[q < 0.9]
    # soft tissue around 1000-1200 with noise sigma 30, and bone shells at 2500-3500
    assert 0.6 < np.mean((body > 850) & (body < 1350)) < 1.0
    assert np.any(body > 2400) and np.all(body < 3500 + 6 * 30)
    assert w["grad"] == "zucker_hummel" and w["skip_empty"]


def test_ellipsoids_and_batch_recipes():
    w = P.workload_ellipsoids_256()
    v = w["volume"]
    assert v.shape == (256, 256, 256) and v.dtype == np.uint16 and v.max() <= 4095
    assert (w["camera"]["width"], w["camera"]["height"]) == (1024, 1024)
    assert w["grad"] == "sobel3d"
    # noise everywhere: no flat region larger than a few voxels away from the clamps
    mid = v[100:110, 100:110, 100:110].astype(np.float64)
    assert mid.std() > 5
    b = P.workload_batch(scale=0.25, cams_per_volume=2, size=64)
    assert len(b) == 8
    assert [x["volume"].dtype for x in b] == [np.uint8, np.uint16] * 4
    assert all(len(x["cameras"]) == 2 for x in b)
