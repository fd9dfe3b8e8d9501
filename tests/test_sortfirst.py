"""Sort-first (image-space) multi-GPU rendering and training, host side, on the CPU.

Rays are independent (§2.2, §6), so a frame splits by rows and training splits by views.
Checked here without a GPU: the row partitions cover every row once and share the busy
rows evenly; two gloo ranks that each render their rows (a stand-in renderer that writes a
known function of the pixel) gather and stitch the whole frame on both ranks; two ranks
that each differentiate their views all-reduce their gradients to the sum over all views.
The GPU side -- the bands rendered by the library stitch to the whole frame bit for bit --
is tests/test_gpu_sortfirst.py.
"""
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

from paper_1609_01317_gb300 import sortfirst as SF  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("H,world,busy", [(1080, 2, (300, 800)), (1080, 8, (0, 1080)),
                                          (37, 5, (10, 12)), (16, 3, None), (5, 8, (1, 4))])
def test_bands_cover_every_row_once_and_share_the_busy_rows(H, world, busy):
    b = SF.bands(H, world, busy)
    assert len(b) == world
    rows = [r for a, c in b for r in range(a, c)]
    assert rows == list(range(H))
    y0, y1 = busy if busy else (0, H)
    share = [len(set(range(a, c)) & set(range(y0, y1))) for a, c in b]
    assert max(share) - min(share) <= 1


@pytest.mark.parametrize("H,world,rows", [(1080, 3, 16), (100, 8, 7), (5, 4, 16)])
def test_stripes_cover_every_row_once(H, world, rows):
    s = SF.stripes(H, world, rows)
    got = sorted(r for per in s for a, c in per for r in range(a, c))
    assert got == list(range(H))
    P = SF.RowPartition(H, 4, s)
    assert P.capacity == max(sum(c - a for a, c in per) for per in s)


def test_partition_rejects_gaps_and_overlaps():
    with pytest.raises(ValueError):
        SF.RowPartition(10, 4, [[(0, 5)], [(6, 10)]])
    with pytest.raises(ValueError):
        SF.RowPartition(10, 4, [[(0, 6)], [(5, 10)]])


def _fake_frame(H, W):
    """The frame a stand-in renderer produces: a known, distinct value per pixel and channel."""
    y, x, c = np.meshgrid(np.arange(H), np.arange(W), np.arange(4), indexing="ij")
    return torch.from_numpy((y * 1000.0 + x + c * 0.25).astype(np.float32))


def _rank_render(rank, world, port, kind, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        H, W = 45, 7
        full = _fake_frame(H, W)
        if kind == "bands":
            P = SF.RowPartition.from_bands(H, W, world, busy=(9, 40))
        else:
            P = SF.RowPartition.from_stripes(H, W, world, rows=4)
        calls = []

        def render_rows(a, b, dst):
            calls.append((a, b))
            dst.copy_(full[a:b])  # this rank's rows only

        packed = torch.full((P.capacity, W, 4), float("nan"))
        P.render_local(rank, render_rows, packed)
        frame = P.gather(packed, torch.empty((H, W, 4)))
        out[rank] = (bool(torch.equal(frame, full)), calls)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["bands", "stripes"])
def test_two_ranks_render_their_rows_and_stitch_the_frame(kind):
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_render, args=(r, world, port, kind, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    rendered = []
    for r in range(world):
        ok, calls = out[r]
        assert ok  # every rank holds the whole frame
        rendered += [row for a, b in calls for row in range(a, b)]
    assert sorted(rendered) == list(range(45))  # each row rendered by exactly one rank


def _view_grad(v, n=6):
    """Stand-in gradient of view v's loss with respect to an n^3 volume and an 8 x 4 table."""
    g = np.random.default_rng(100 + v)
    return (torch.from_numpy(g.standard_normal((n, n, n)).astype(np.float32)),
            torch.from_numpy(g.standard_normal((8, 4)).astype(np.float32)))


def _rank_train(rank, world, port, nviews, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = SF.view_share(nviews, world, rank)
        gv = torch.zeros((6, 6, 6))
        gt = torch.zeros((8, 4))
        for v in mine:  # this rank's views, accumulated as vr_render_backward_views does
            a, b = _view_grad(v)
            gv += a
            gt += b
        SF.allreduce_gradients([gv, gt, None])
        out[rank] = (mine, gv.numpy(), gt.numpy())
    finally:
        dist.destroy_process_group()


def test_two_ranks_sum_their_views_gradients():
    world, nviews = 2, 16
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_train, args=(r, world, port, nviews, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want_v = sum(_view_grad(v)[0] for v in range(nviews)).numpy()
    want_t = sum(_view_grad(v)[1] for v in range(nviews)).numpy()
    assert sorted(out[0][0] + out[1][0]) == list(range(nviews))
    for r in range(world):
        np.testing.assert_allclose(out[r][1], want_v, rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(out[r][2], want_t, rtol=1e-5, atol=1e-5)
    # both ranks hold bit-identical sums, so their optimiser steps stay identical
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def test_view_share():
    assert SF.view_share(16, 3, 0) == [0, 3, 6, 9, 12, 15]
    assert sorted(sum((SF.view_share(16, 3, r) for r in range(3)), [])) == list(range(16))
    with pytest.raises(ValueError):
        SF.view_share(4, 2, 2)
