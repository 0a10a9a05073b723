"""Autotuner for the FP32 launch shapes of the step kernels: the strip height
of a grid's step (16, 32 or 64 rows) and of a patch level's step (16 or 32
rows).

The launch shape changes only throughput, never results.  The tuner times
each candidate with CUDA events on a few steps and keeps the faster one,
caching the choice per shape signature (grid size, or the histogram of patch
sizes of a level) for the life of the process.

Tuning steps the object it is given: tune before setting the state you want
to keep (or set it again afterwards; patch levels must be restarted).
"""
from __future__ import annotations

from . import swadj as S

CANDIDATES = (32, 16)         # patch-level strip heights
GRID_CANDIDATES = (32, 16, 64)  # grid strip heights
_cache: dict = {}


def _time(fn, steps):
    import torch
    fn(2)  # warm up (first launch sets kernel attributes)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    fn(steps)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune_grid(grid: "S.Grid", steps: int = 10) -> int:
    """Pick the strip height for a FP32 grid; returns it and applies it."""
    key = ("grid", grid.desc.nx, grid.desc.ny)
    if key not in _cache:
        best, best_t = None, None
        for rows in GRID_CANDIDATES:
            S.swa_grid_set_strip_rows(grid.h, rows)
            t = _time(lambda n: grid.step(n, 1e300), steps)
            if best_t is None or t < best_t:
                best, best_t = rows, t
        _cache[key] = best
    S.swa_grid_set_strip_rows(grid.h, _cache[key])
    return _cache[key]


def _level_signature(ps: "S.PatchSet", level: int):
    sizes = sorted((p[3], p[4]) for p in ps.patches if p[0] == level)
    hist = {}
    for nx, ny in sizes:
        b = (min(nx // 32, 8), min(ny // 16, 16))
        hist[b] = hist.get(b, 0) + 1
    return ("patches", level, tuple(sorted(hist.items())))


def tune_patches(ps: "S.PatchSet", steps: int = 5) -> dict:
    """Pick the strip height of every level of a patch set (levels must have
    been started); returns {level: rows} and applies it."""
    out = {}
    for level in ps.levels:
        key = _level_signature(ps, level)
        if key not in _cache:
            best, best_t = None, None
            for rows in CANDIDATES:
                S.swa_patches_set_tile_rows(ps.h, level, rows)
                t = _time(lambda n: ps.step(level, n), steps)
                if best_t is None or t < best_t:
                    best, best_t = rows, t
            _cache[key] = best
        S.swa_patches_set_tile_rows(ps.h, level, _cache[key])
        out[level] = _cache[key]
    return out
