"""Autotuner for the FP32 launch shapes of the step kernels: the strip height
of a grid's step (16, 32 or 64 rows) and of a patch level's step (16 or 32
rows).

The launch shape changes only throughput, never results.  The tuner times
each candidate with CUDA events on a few steps and keeps the faster one.  The
choice is cached per device and shape signature (grid size, or the histogram
of patch sizes of a level), in the process and in a JSON file that later
processes read back (SWA_TUNE_CACHE names the file; the default lives in the
user's cache directory; SWA_TUNE_CACHE="" keeps the cache in the process).

Tuning steps the object it is given: tune before setting the state you want
to keep (or set it again afterwards; patch levels must be restarted).
"""
from __future__ import annotations

import json
import os

from . import swadj as S

CANDIDATES = (32, 16)         # patch-level strip heights
GRID_CANDIDATES = (32, 16, 64)  # grid strip heights
_cache: dict = {}
_loaded_from = None


def cache_path():
    """The cache file, or None for a cache in the process only."""
    p = os.environ.get("SWA_TUNE_CACHE")
    if p is not None:
        return p or None
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1605_05320_gb300",
                        "tune.json")


def _key(key) -> str:
    return json.dumps(key, separators=(",", ":"))


def _load():
    global _loaded_from
    path = cache_path()
    if path == _loaded_from:
        return
    _loaded_from = path
    if path and os.path.exists(path):
        try:
            with open(path) as fh:
                data = json.load(fh)
            if isinstance(data, dict):
                for k, v in data.items():
                    if isinstance(v, int):
                        _cache.setdefault(k, v)
        except (OSError, ValueError):
            pass   # an unreadable cache is only a cache: tune again


def _store():
    path = cache_path()
    if not path:
        return
    try:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(_cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _device():
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


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


def _choose(key, candidates, apply, run, steps):
    _load()
    k = _key(key)
    if k not in _cache:
        best, best_t = None, None
        for rows in candidates:
            apply(rows)
            t = _time(run, steps)
            if best_t is None or t < best_t:
                best, best_t = rows, t
        _cache[k] = best
        _store()
    apply(_cache[k])
    return _cache[k]


def tune_grid(grid: "S.Grid", steps: int = 10) -> int:
    """Pick the strip height for a FP32 grid; returns it and applies it."""
    key = [_device(), "grid", grid.desc.nx, grid.desc.ny]
    return _choose(key, GRID_CANDIDATES, lambda rows: S.swa_grid_set_strip_rows(grid.h, rows),
                   lambda n: grid.step(n, 1e300), steps)


def _level_signature(ps: "S.PatchSet", level: int):
    sizes = sorted((p[3], p[4]) for p in ps.patches if p[0] == level)
    hist = {}
    for nx, ny in sizes:
        b = (min(nx // 32, 8), min(ny // 16, 16))
        hist[b] = hist.get(b, 0) + 1
    return ["patches", level, sorted([list(b), c] for b, c in hist.items())]


def tune_patches(ps: "S.PatchSet", steps: int = 5) -> dict:
    """Pick the strip height of every level of a patch set (levels must have
    been started); returns {level: rows} and applies it."""
    out = {}
    for level in ps.levels:
        key = [_device()] + _level_signature(ps, level)
        out[level] = _choose(key, CANDIDATES,
                             lambda rows, lv=level: S.swa_patches_set_tile_rows(ps.h, lv, rows),
                             lambda n, lv=level: ps.step(lv, n), steps)
    return out
