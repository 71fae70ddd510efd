"""Splitting one volume into z-slabs (the paper's parallelisation over vertex subsets,
Section 5.3).

A volume too large for one device is cut along its slowest axis (z, axis 2) into slabs
of consecutive planes.  Each slab's pixel buffer also holds the plane on each side that
exists (the lower-star stencil of a boundary vertex reads it; the neighbouring slab owns
it).  Each device builds the tables of its slab (``tables_create_slab``) and evaluates
the transforms of the slab's part; since every transform is a sum over vertices
(Lemma 3.1), the parts add up to the volume's transform.  The exchange is one gather of
the parts in slab order followed by ``slab_sum`` on the device (exact integer sums for
ECT and Radon, compensated FP64 sums for the hybrid transforms).

This module only splits, packs and exchanges: every sum runs in the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding


def slab_bounds(depth: int, parts: int) -> list:
    """Balanced contiguous plane ranges [(z0, z1), ...] covering [0, depth)."""
    if parts < 1 or depth < parts:
        raise ValueError("need 1 <= parts <= depth")
    cuts = [(depth * p) // parts for p in range(parts + 1)]
    return [(cuts[p], cuts[p + 1]) for p in range(parts)]


def buffer_planes(z0: int, z1: int, depth: int) -> tuple:
    """Planes a slab's pixel buffer holds: [max(z0 - 1, 0), min(z1 + 1, depth))."""
    return max(z0 - 1, 0), min(z1 + 1, depth)


def pack_slabs(volume: np.ndarray, ranges, device="cuda", align: int = 16):
    """Pixel buffer of the slabs `ranges` of one volume (numpy [m2, m1, m0], axis 0 of the
    library = the last numpy axis), for one handle with one image per slab.

    Returns (pixels, shapes, offsets, zrange) as tables_create_slab and Tables.build take
    them; every image's shape is the whole volume's."""
    if volume.ndim != 3:
        raise ValueError("slabs split 3-D volumes")
    m2, m1, m0 = volume.shape
    chunks, offsets, off = [], [], 0
    for z0, z1 in ranges:
        lo, hi = buffer_planes(z0, z1, m2)
        part = np.ascontiguousarray(volume[lo:hi]).reshape(-1)
        pad = (-off) % align
        if pad:
            chunks.append(np.zeros(pad, dtype=volume.dtype))
            off += pad
        offsets.append(off)
        chunks.append(part)
        off += part.size
    pixels = torch.from_numpy(np.concatenate(chunks)).to(device)
    shapes = np.array([[m0, m1, m2]] * len(ranges), dtype=np.int64)
    zrange = np.array(list(ranges), dtype=np.int64)
    return pixels, shapes, np.array(offsets, dtype=np.int64), zrange


def build_slab_tables(volume: np.ndarray, ranges, device="cuda", stream=None) -> binding.Tables:
    """Tables of the slabs `ranges` of `volume` (one image per slab), built and synced."""
    pixels, shapes, offsets, zrange = pack_slabs(volume, ranges, device)
    dtype = binding.U8 if pixels.dtype == torch.uint8 else binding.I32
    t = binding.tables_create_slab(shapes, offsets, zrange, dtype)
    t.build(pixels, stream)
    t.sync(stream)
    t._pixels = pixels   # keep the buffer alive as long as the handle
    return t


def gather_parts(local: torch.Tensor, group=None) -> torch.Tensor:
    """Every rank's part, stacked in rank order: [world, *local.shape] (communication only)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local.contiguous(), group=group)
    return torch.stack(parts)


def reduce_slabs(local: torch.Tensor, group=None) -> torch.Tensor:
    """The volume's transform from this rank's slab part: gather in rank order, then the
    library's slab sum (exact for int32, compensated for float64) on this rank's device."""
    return binding.slab_sum(gather_parts(local, group))
