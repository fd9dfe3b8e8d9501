"""Sort-last (object-space) multi-GPU rendering, host side, on the CPU.

The volume splits into z slabs; each rank composites the samples of its slab into a
premultiplied partial image and the partial images combine with "over", front to back
along each pixel's ray (Eq. 6 is associative). Checked here without a GPU: the slabs cover
every z once in whole bricks; the per-pixel order follows the ray's direction in z; the
composite equals a plain per-pixel front-to-back loop over the slabs; two gloo ranks that
each hold one slab's partial image gather and composite the same image on both ranks. The
GPU side -- the library's partial images composite to the whole frame -- is
tests/test_gpu_sortlast.py.
"""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import phantoms as P  # noqa: E402
from paper_1609_01317_gb300 import sortlast as SL  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("nz,world", [(361, 2), (361, 8), (64, 3), (9, 4), (8, 5), (1, 1)])
def test_slabs_cover_every_z_once_in_whole_bricks(nz, world):
    s = SL.zslabs(nz, world)
    assert len(s) == world
    assert s[0][0] == -math.inf and s[-1][1] == math.inf
    for (a0, a1), (b0, b1) in zip(s, s[1:]):
        assert a1 == b0 and a0 <= a1
    inner = [z for z, _ in s[1:]]
    assert all(z % 8 == 0 for z in inner)
    nb = (nz + 7) // 8
    bricks = [int((min(b, 8 * nb) - max(a, 0)) // 8) for a, b in s]
    assert max(bricks) - min(bricks) <= 1 and sum(bricks) == nb


def _partials(H, W, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        a = rng.uniform(0.0, 0.9, (H, W, 1))
        c = rng.uniform(0.0, 1.0, (H, W, 3)) * a  # premultiplied
        out.append(torch.from_numpy(np.concatenate([c, a], axis=2).astype(np.float32)))
    return out


def _loop_composite(parts, sign):
    """Per pixel: the slabs in ray order, each folded in with 'over'."""
    H, W, _ = parts[0].shape
    out = np.zeros((H, W, 4))
    for y in range(H):
        for x in range(W):
            order = range(len(parts)) if sign[y, x] > 0 else range(len(parts) - 1, -1, -1)
            c, a = np.zeros(3), 0.0
            for i in order:
                p = parts[i][y, x].double().numpy()
                c = c + (1.0 - a) * p[:3]
                a = a + (1.0 - a) * p[3]
            out[y, x, :3], out[y, x, 3] = c, a
    return out


def test_composite_is_the_front_to_back_over_in_each_pixels_order():
    H, W = 6, 9
    parts = _partials(H, W, 4, 3)
    sign = np.where(np.arange(H * W).reshape(H, W) % 3 == 0, -1, 1).astype(np.int8)
    got = SL.composite(parts, sign).double().numpy()
    np.testing.assert_allclose(got, _loop_composite(parts, sign), rtol=0, atol=2e-6)
    # one slab is the identity; transparent slabs change nothing
    np.testing.assert_array_equal(SL.composite(parts[:1], sign).numpy(), parts[0].numpy())
    zero = torch.zeros_like(parts[0])
    np.testing.assert_allclose(SL.composite([zero, parts[1], zero], sign).numpy(),
                               parts[1].numpy(), atol=0)


def test_ray_dz_sign_follows_the_rays():
    # orthographic from below: every ray moves towards +z; from above: towards -z
    shp = (40, 30, 20)
    below = P.orbit_camera(shp, 8, 6, 0.3, -1.2, ortho=True, ortho_height=50.0)
    above = P.orbit_camera(shp, 8, 6, 0.3, 1.2, ortho=True, ortho_height=50.0)
    assert (SL.ray_dz_sign(below) == 1).all() and (SL.ray_dz_sign(above) == -1).all()
    # a perspective eye at mid height looking along +x: the upper rows rise, the lower fall
    cam = P.camera((-50.0, 15.0, 10.0), (20.0, 15.0, 10.0), (0.0, 0.0, 1.0), 16, 12,
                   fov_y_deg=60.0)
    s = SL.ray_dz_sign(cam)
    assert (s[:6] == 1).all() and (s[6:] == -1).all()


def _rank_composite(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        H, W = 5, 7
        parts = _partials(H, W, world, 11)  # every rank can build all; each renders its own
        sign = np.where(np.arange(H * W).reshape(H, W) % 2 == 0, 1, -1).astype(np.int8)
        part = SL.SlabPartition(16 * world, world)
        mine = torch.empty((H, W, 4))
        part.render_local(rank, lambda z0, z1, dst: dst.copy_(parts[rank]), mine)
        frame = part.gather(mine, sign)
        out[rank] = frame.numpy().tobytes()
        if rank == 0:
            out["ref"] = SL.composite(parts, sign).numpy().tobytes()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_and_composite_the_same_image():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_composite, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == out["ref"]
