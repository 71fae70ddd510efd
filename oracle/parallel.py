"""The oracle run over several host processes, as the paper parallelises (Section 5.3).

TEST INFRASTRUCTURE ONLY: used by bench.py's CPU baseline (and the reference arm) to
time the oracle on the host's cores; never by the product path.

Tables are split over vertices: row blocks of a 2-D image, each computed from its rows
plus a one-row halo on each side whose own (boundary-distorted) values are dropped, so
that the blocks' entries, concatenated in block order, are the whole image's tables.
Transforms are split over directions; workers read the tables from memory-mapped .npy
files written once by the parent.
"""
from __future__ import annotations

import time

import numpy as np

from . import oracle as O

_TABLES = None


def block_tables(args):
    """Non-zero (global index, value) pairs of the 2^n lower tables and the 2^(n-1) Delta
    tables of image rows [r0, r0 + count), from `rows` = image rows [r0 - skip, ...) that
    include the halo."""
    rows, skip, count, r0 = args
    low = O.lower_star_values(rows)[:, skip:skip + count]
    d = O.delta_values(low)
    W = rows.shape[1]
    out = []
    for arr in list(low) + list(d):
        flat = arr.reshape(-1)
        idx = np.flatnonzero(flat)
        out.append((idx + r0 * W, flat[idx]))
    return out


def row_blocks(img: np.ndarray, parts: int):
    """Arguments of block_tables for `parts` row blocks of a 2-D image."""
    H = img.shape[0]
    out = []
    for i in range(parts):
        r0, r1 = (H * i) // parts, (H * (i + 1)) // parts
        lo, hi = max(r0 - 1, 0), min(r1 + 1, H)
        out.append((img[lo:hi], r0 - lo, r1 - r0, r0))
    return out


def merge_blocks(shape, parts) -> O.CriticalTables:
    """The tables of the whole image from the blocks' entries (in block order)."""
    t = O.CriticalTables(shape=tuple(shape))
    n = len(shape)
    NO = 1 << n
    for s in range(NO + NO // 2):
        idx = np.concatenate([p[s][0] for p in parts]).astype(np.int64)
        val = np.concatenate([p[s][1] for p in parts]).astype(np.int64)
        (t.lower_idx if s < NO else t.delta_idx).append(idx)
        (t.lower_val if s < NO else t.delta_val).append(val)
    t.chi = int(t.lower_val[0].sum())
    return t


def worker_init(paths, shape, chi):
    """Pool initializer: the tables from the .npy files (idx, val per table, in order)."""
    global _TABLES
    t = O.CriticalTables(shape=tuple(shape))
    NO = 1 << len(shape)
    arrs = [np.load(p, mmap_mode="r") for p in paths]
    for s in range(NO + NO // 2):
        (t.lower_idx if s < NO else t.delta_idx).append(arrs[2 * s])
        (t.lower_val if s < NO else t.delta_val).append(arrs[2 * s + 1])
    t.chi = chi
    _TABLES = t


def transform_task(args):
    """One worker's share of a transform: ("ect" | "radon", dirs, a, b, T) or
    ("ht", dirs, kernels).  Returns (seconds, hybrid terms evaluated)."""
    what, dirs = args[0], args[1]
    t = _TABLES
    t0 = time.time()
    terms = 0
    if what == "ect":
        O.ect_grid(t, dirs, *args[2:5])
    elif what == "radon":
        O.radon_grid(t, dirs, *args[2:5])
    else:
        half = 1 << (t.n - 1)
        for k in args[2]:
            O.hybrid_transform(t, k, dirs)
            for xi in dirs:
                o = O.orthant_of(xi)
                terms += len(t.delta_idx[o if o < half else O.partner(o, t.n)])
    return time.time() - t0, terms
