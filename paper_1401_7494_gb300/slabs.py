"""z-slab sharding of one reconstruction over several GPUs.

Every voxel's sum is independent of every other voxel's, and the paper
parallelises the backprojection over voxel planes (Section "Implementation").
Across GPUs the same split gives each rank a contiguous slab of z planes: the
rank reads every projection and every matrix but holds and updates only its
own planes (``rct_create_slab``), so the passes exchange nothing.  The one
exchange is the read-back, when the slabs are brought together into one
volume (``gather_slabs``); a caller that keeps the slabs where they are skips
it.

Slab boundaries are multiples of 16 planes, the longest z-run of the
kernels, so every z-run of a slab is the z-run the whole-volume context
would use and the result is bit for bit the whole-volume result.
"""
from __future__ import annotations

from dataclasses import dataclass

ALIGN = 16          # planes: every z-run length of the kernels divides it


def slab_ranges(L: int, parts: int, align: int = ALIGN) -> list[tuple[int, int]]:
    """Split planes [0, L) into ``parts`` contiguous (z_first, z_count) slabs.

    Boundaries fall on multiples of ``align`` (the last slab ends at L); the
    blocks of ``align`` planes are dealt out as evenly as possible, earlier
    slabs taking the extra block.  A slab can be empty (z_count 0) only when
    there are fewer blocks than parts."""
    if L <= 0 or parts <= 0 or align <= 0:
        raise ValueError(f"L={L}, parts={parts}, align={align} must be positive")
    blocks = -(-L // align)
    base, extra = divmod(blocks, parts)
    out = []
    b = 0
    for r in range(parts):
        nb = base + (1 if r < extra else 0)
        z0 = min(b * align, L)
        z1 = min((b + nb) * align, L)
        out.append((z0, z1 - z0))
        b += nb
    return out


@dataclass
class SlabPlan:
    """Rank ``rank`` of ``world`` holds planes [z_first, z_first + z_count) of an L^3 volume."""
    L: int
    rank: int
    world: int
    z_first: int
    z_count: int
    align: int = ALIGN

    @classmethod
    def for_rank(cls, L: int, rank: int, world: int, align: int = ALIGN) -> "SlabPlan":
        if not 0 <= rank < world:
            raise ValueError(f"rank {rank} outside [0, {world})")
        z0, zc = slab_ranges(L, world, align)[rank]
        return cls(L, rank, world, z0, zc, align)

    @property
    def empty(self) -> bool:
        return self.z_count == 0

    @property
    def updates_per_view(self) -> int:
        return self.z_count * self.L * self.L


def gather_slabs(local, plan: SlabPlan, dst=None, dist=None, group=None):
    """Bring the ranks' slabs together on rank 0 (the read-back of a sharded reconstruction).

    ``local`` is this rank's slab, a tensor of z_count x L x L floats (on the device of
    the rank's backend: CUDA for NCCL, host for gloo).  Rank 0 passes ``dst``, an
    L x L x L tensor on the same kind of device, and receives every other rank's
    planes into it point to point; the other ranks send theirs.  Returns ``dst`` on
    rank 0 and None elsewhere.  ``dist`` is ``torch.distributed`` (initialised)."""
    import torch
    if dist is None:
        import torch.distributed as dist
    if tuple(local.shape) != (plan.z_count, plan.L, plan.L):
        raise ValueError(f"local slab has shape {tuple(local.shape)}, expected {(plan.z_count, plan.L, plan.L)}")
    ranges = slab_ranges(plan.L, plan.world, plan.align)
    if plan.rank != 0:
        if plan.z_count:
            dist.send(local.contiguous(), dst=0, group=group)
        return None
    if dst is None or tuple(dst.shape) != (plan.L,) * 3:
        raise ValueError("rank 0 needs an L x L x L destination")
    z0, zc = ranges[0]
    if zc:
        dst[z0:z0 + zc].copy_(local)
    for r in range(1, plan.world):
        z0, zc = ranges[r]
        if zc:
            buf = torch.empty((zc, plan.L, plan.L), dtype=local.dtype, device=local.device)
            dist.recv(buf, src=r, group=group)
            dst[z0:z0 + zc].copy_(buf)
    return dst


class SlabBackprojector:
    """A rank's part of a sharded reconstruction: a slab context on the current device.

    ``bp`` is an ``rct.Backprojector`` over the rank's planes, with the usual calls
    (geometry, precision, tuning, reset, backproject, read-back); every projection goes to
    every rank, each rank adds it into its own planes only.  Every rank must hold at least
    one block of planes (L >= 16 * world)."""

    def __init__(self, L: int, det_w: int, det_h: int, n_views: int, rank: int, world: int,
                 align: int = ALIGN):
        from . import rct
        self.plan = SlabPlan.for_rank(L, rank, world, align)
        if self.plan.empty:
            raise ValueError(f"L={L} has fewer {align}-plane blocks than the {world} ranks: rank {rank} holds none")
        self.bp = rct.Backprojector(L, det_w, det_h, n_views, z_range=(self.plan.z_first, self.plan.z_count))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self.bp is not None:
            self.bp.close()
            self.bp = None
