"""Sort-first (image-space) multi-GPU rendering and training.

Rays are independent (§2.2; §6 suggests spreading them over several processors), so a frame
splits by pixels with no exchange during the march: every GPU holds the same volume and
transfer function, renders its rows of the frame with ``vr_render_rows`` and the rows are
gathered (one all-gather of the image).  Training splits by views: each GPU renders and
differentiates its share of the views, and the volume and table gradients are summed over
the GPUs (one all-reduce), after which every GPU takes the same optimiser step on identical
parameters.

Collectives go through ``torch.distributed`` (NCCL between GPUs; the host-side logic is
tested with gloo on the CPU).  Everything that decides which rank owns which rows or views is
plain host arithmetic here; the rendering itself is the library's.
"""
from __future__ import annotations

__all__ = ["bands", "stripes", "RowPartition", "view_share", "allreduce_gradients"]


def bands(height: int, world: int, busy=None):
    """Contiguous row bands, one per rank: [(row0, row1)] * world covering [0, height).

    ``busy`` = (y0, y1), the rows where rays can meet the volume (its screen rectangle,
    ``vr_screen_rect``): those rows are shared as evenly as possible and the rows above and
    below, whose rays miss the volume, go to the first and the last band.  A rank may get an
    empty band when there are more ranks than busy rows."""
    if world < 1 or height < 0:
        raise ValueError("world >= 1 and height >= 0 required")
    y0, y1 = (0, height) if busy is None else (max(0, int(busy[0])), min(height, int(busy[1])))
    if y1 < y0:
        y0 = y1 = 0
    n = y1 - y0
    cuts = [y0 + (n * r) // world for r in range(world + 1)]
    cuts[0], cuts[-1] = 0, height
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def stripes(height: int, world: int, rows: int = 16):
    """Stripes of ``rows`` rows dealt round-robin: stripe i goes to rank i % world.  Returns,
    per rank, its list of (row0, row1).  Interleaving evens out the cost of a frame whose
    busy rows sit in the middle of the image, at one render call per stripe."""
    if world < 1 or rows < 1:
        raise ValueError("world >= 1 and rows >= 1 required")
    out = [[] for _ in range(world)]
    for i, r0 in enumerate(range(0, height, rows)):
        out[i % world].append((r0, min(height, r0 + rows)))
    return out


class RowPartition:
    """Which rows of an H x W frame each rank renders, and how the gathered rows are put
    back together.  ``per_rank[r]`` is rank r's list of (row0, row1); every rank packs its
    rows, in that order, into a buffer of ``capacity`` rows (the largest share), so that one
    equal-sized all-gather moves every rank's rows."""

    def __init__(self, height: int, width: int, per_rank):
        self.height, self.width = int(height), int(width)
        self.per_rank = [list(map(tuple, p)) for p in per_rank]
        rows = sorted(r for p in self.per_rank for (a, b) in p for r in range(a, b))
        if rows != list(range(self.height)):
            raise ValueError("the partition must cover every row exactly once")
        self.capacity = max(1, max(sum(b - a for a, b in p) for p in self.per_rank))

    @classmethod
    def from_bands(cls, height, width, world, busy=None):
        return cls(height, width, [[b] if b[1] > b[0] else [] for b in bands(height, world, busy)])

    @classmethod
    def from_stripes(cls, height, width, world, rows=16):
        return cls(height, width, stripes(height, world, rows))

    @property
    def world(self) -> int:
        return len(self.per_rank)

    def render_local(self, rank: int, render_rows, packed):
        """Fill ``packed`` (capacity x W x 4) with rank's rows: ``render_rows(row0, row1, out)``
        writes rows [row0, row1) into ``out`` (a (row1 - row0) x W x 4 view of ``packed``)."""
        at = 0
        for a, b in self.per_rank[rank]:
            render_rows(a, b, packed[at:at + (b - a)])
            at += b - a
        return packed

    def stitch(self, gathered, out):
        """Scatter every rank's packed rows (gathered[r], capacity x W x 4) into the frame
        ``out`` (H x W x 4); returns ``out``."""
        for r, rows in enumerate(self.per_rank):
            at = 0
            for a, b in rows:
                out[a:b] = gathered[r][at:at + (b - a)]
                at += b - a
        return out

    def gather(self, packed, out, group=None):
        """All-gather the ranks' packed rows and stitch the whole frame into ``out`` on every
        rank (torch.distributed; NCCL for CUDA tensors, gloo for CPU tensors)."""
        import torch
        import torch.distributed as dist

        if self.world == 1:
            return self.stitch([packed], out)  # one rank: nothing to exchange
        parts = [torch.empty_like(packed) for _ in range(self.world)]
        dist.all_gather(parts, packed, group=group)
        return self.stitch(parts, out)


def view_share(nviews: int, world: int, rank: int):
    """The views rank ``rank`` renders and differentiates in a training step: round-robin,
    so every rank gets nviews / world of them (one more for the first nviews % world)."""
    if not 0 <= rank < world:
        raise ValueError("0 <= rank < world required")
    return list(range(rank, nviews, world))


def allreduce_gradients(tensors, group=None):
    """Sum the volume and transfer-function gradients (and anything else given) over the
    ranks in place: after it every rank holds the gradient of the whole loss."""
    import torch.distributed as dist

    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors
