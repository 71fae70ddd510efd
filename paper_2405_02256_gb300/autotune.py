"""Autotuner of the evaluation tile shapes (directions per warp/lane, points per work
item, resident blocks per SM), with a JSON cache keyed by GPU, operation and size.

Each candidate is timed with CUDA events on the current stream (median of a few
launches after a warm-up); the fastest is set on the tables handle and stored in the
cache so that later processes pick it up without timing.  Results do not depend on the
tile shapes except for the rounding order of hybrid transforms, which stays within the
documented accuracy.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import binding as tb

CACHE = os.environ.get("TOPOT_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json"))

ECT_SPACE = [dict(ect_dirs_per_warp=td, ect_chunk=ch, ect_ctas_per_sm=c)
             for td in (8, 16, 32, 64) for ch in (0, 16384, 131072) for c in (0, 1)]
HT_SPACE = [dict(ht_dirs_per_lane=dl, ht_chunk=ch, ht_ctas_per_sm=c, ht_warp_split=sp)
            for dl in (1, 2, 4, 8) for ch in (0, 16384, 131072) for c in (0, 3) for sp in (1, 2)
            if sp == 1 or dl in (2, 4)]


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(cache: dict):
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _key(tables: tb.Tables, op: str, D: int, extra: str) -> str:
    gpu = torch.cuda.get_device_name()
    vox = int(sum(int(math.prod(s)) for s in tables.shapes))
    bucket = f"B{2 ** int(math.log2(max(1, tables.B)))}_V{2 ** int(math.log2(max(1, vox)))}_D{2 ** int(math.log2(max(1, D)))}"
    return f"{gpu}|n{tables.n}|{op}|{extra}|{bucket}"


def _time(fn, reps: int = 3) -> float:
    fn()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sorted(ts)[len(ts) // 2]


def tune(tables: tb.Tables, op: str, dirs: torch.Tensor, *, kernel: str = "laplace", precision: str = "fp32c",
         t_min: float = -1.0, t_max: float = 1.0, T: int = 64, use_cache: bool = True, space=None) -> dict:
    """Pick and set the fastest tile shapes of ``op`` ('ect', 'radon' or 'hybrid')."""
    D = dirs.shape[-2]
    extra = f"{kernel}-{precision}" if op == "hybrid" else f"T{T}"
    key = _key(tables, op, D, extra)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        tables.set_tuning(**cache[key]["tuning"])
        return cache[key]
    if op == "hybrid":
        space = space or [c for c in HT_SPACE if not (c["ht_dirs_per_lane"] == 8 and kernel != "laplace")]
        if precision == "fp64":
            space = [c for c in space if c["ht_dirs_per_lane"] == 1]
        out = torch.empty((tables.B, D, 2) if kernel == "fourier" else (tables.B, D), dtype=torch.float64,
                          device=dirs.device)

        def run():
            tb.hybrid_transform(tables, kernel, dirs, precision, out=out)
    else:
        space = space or ECT_SPACE
        out = torch.empty((tables.B, D, T), dtype=torch.int32, device=dirs.device)
        f = tb.ect if op == "ect" else tb.radon

        def run():
            f(tables, dirs, t_min, t_max, T, out=out)
    best = None
    for cand in space:
        try:
            tables.set_tuning(**cand)
            ms = _time(run)
        except tb.TopotError:
            continue
        if best is None or ms < best["ms"]:
            best = {"tuning": dict(cand), "ms": ms}
    tables.set_tuning(**best["tuning"])
    if use_cache:
        cache = _load_cache()
        cache[key] = best
        _save_cache(cache)
    return best
