"""Sort-last (object-space) multi-GPU rendering.

The volume is split into slabs along z, one per rank; every rank marches the whole frame but
composites only the samples inside its slab (``vr_render_partial``: the whole sampling box's
grid of samples, so the slabs' samples are exactly the frame's), giving a premultiplied
partial image (C, A).  Eq. 6 (§3.9) is associative, so the partial images combine pixel by
pixel with "over", front to back along the pixel's ray:

    C = C_front + (1 - A_front) C_back,   A = A_front + (1 - A_front) A_back,

which is the whole frame up to rounding when early termination is off (each slab marches
all of its samples).  The order of the slabs along a ray is that of increasing z where the
ray's direction has d_z > 0 and of decreasing z where d_z < 0, so one frame can hold both
orders (an eye within the volume's z range).  The partial images are exchanged with one
all-gather and composited on every rank.

Collectives go through ``torch.distributed`` (NCCL between GPUs; the host-side logic is
tested with gloo on the CPU).
"""
from __future__ import annotations

import math

__all__ = ["zslabs", "ray_dz_sign", "composite", "SlabPartition"]


def zslabs(nz: int, world: int, brick: int = 8):
    """Contiguous z ranges, one per rank, splitting the volume's depth [0, nz - 1] in whole
    bricks of ``brick`` voxels as evenly as possible; the first starts at -inf and the last
    ends at +inf, so every sample of the box (rounding included) lies in exactly one.
    A rank gets an empty range ((z, z) is returned as (z, z)) when there are more ranks than
    bricks."""
    if world < 1 or nz < 1 or brick < 1:
        raise ValueError("world >= 1, nz >= 1 and brick >= 1 required")
    nb = (nz + brick - 1) // brick
    cuts = [float(brick * ((nb * r) // world)) for r in range(world + 1)]
    cuts[0], cuts[-1] = -math.inf, math.inf
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def ray_dz_sign(cam: dict):
    """Per pixel, +1 where the pixel's ray moves towards +z (or not at all along z), -1
    where it moves towards -z: an (H, W) int8 numpy array.  Computed from the camera as the
    library's ray set-up does (direction = fwd + u right + v up; the normalisation does not
    change its sign)."""
    import numpy as np

    eye = np.asarray(cam["eye"], np.float64)
    tgt = np.asarray(cam["target"], np.float64)
    up = np.asarray(cam["up"], np.float64)
    W, H = int(cam["width"]), int(cam["height"])
    fwd = tgt - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    if cam.get("ortho"):
        dz = np.full((H, W), fwd[2])
    else:
        ay = math.tan(math.radians(float(cam["fov_y_deg"])) / 2.0)
        ax = ay * W / H
        u = ((2.0 * np.arange(W) + 1.0) / W - 1.0) * ax
        v = (1.0 - (2.0 * np.arange(H) + 1.0) / H) * ay
        dz = fwd[2] + u[None, :] * right[2] + v[:, None] * upv[2]
    return np.where(dz < 0.0, -1, 1).astype(np.int8)


def composite(partials, sign, out=None):
    """Composite the partial images (a list of (H, W, 4) tensors, ordered by increasing z)
    front to back per pixel: in list order where ``sign`` (an (H, W) tensor or array of
    +-1) is +1, in reverse order where it is -1.  Returns (H, W, 4) premultiplied (C, A)."""
    import torch

    first = partials[0]
    s = torch.as_tensor(sign, device=first.device).reshape(first.shape[0], first.shape[1], 1)
    fwd = s > 0
    acc = torch.zeros_like(first) if out is None else out.zero_()
    n = len(partials)
    for i in range(n):
        a, b = partials[i], partials[n - 1 - i]
        layer = torch.where(fwd, a, b)  # the i-th slab along each pixel's ray
        t = 1.0 - acc[..., 3:4]
        acc[..., :3] += t * layer[..., :3]
        acc[..., 3:4] += t * layer[..., 3:4]
    return acc


class SlabPartition:
    """Which z slab each rank renders, and how the gathered partial images are composited."""

    def __init__(self, nz: int, world: int, brick: int = 8):
        self.slabs = zslabs(nz, world, brick)

    @property
    def world(self) -> int:
        return len(self.slabs)

    def render_local(self, rank: int, render_partial, out):
        """Rank ``rank``'s partial image into ``out`` with ``render_partial(z0, z1, out)``
        (e.g. ``vr_render_partial`` with the rank's context)."""
        z0, z1 = self.slabs[rank]
        if z0 < z1:
            render_partial(z0, z1, out)
        else:
            out.zero_()
        return out

    def gather(self, partial, sign, out=None, group=None):
        """All-gather every rank's partial image and composite them (on every rank)."""
        import torch
        import torch.distributed as dist

        if self.world == 1:
            return composite([partial], sign, out)  # one rank: nothing to exchange
        parts = [torch.empty_like(partial) for _ in range(self.world)]
        dist.all_gather(parts, partial.contiguous(), group=group)
        return composite(parts, sign, out)
