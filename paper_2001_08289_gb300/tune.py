"""Cache of tuned solve settings, keyed by (grid shape, d, scheme, precision).

The measurement itself is lsfft_autotune in the library (CUDA events on the
grid's stream); this module only remembers its answer in a JSON file so that a
grid shape is tuned once, and applies a stored answer to a grid.
"""
from __future__ import annotations

import json
import os

from . import lsfft_autotune, make_opts


def cache_path() -> str:
    return os.environ.get("LSFFT_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lsfft_gb300", "tune.json"))


def _key(grid, scheme, precision) -> str:
    return f"{'x'.join(str(v) for v in grid.n)}|d{grid.d}|{scheme}|{precision}"


def load(path: str | None = None) -> dict:
    path = path or cache_path()
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def tuned(grid, sigma1, e, path: str | None = None, iters: int = 32, **kw) -> dict:
    """Solve options for `grid` with check_every (and the grid's strided-pass
    layout) taken from the cache, tuning and storing them on a miss.  kw: the
    solve's options as for make_opts; returns them with check_every filled in."""
    path = path or cache_path()
    scheme, precision = kw.get("scheme", "ms"), kw.get("precision", "fp32")
    cache = load(path)
    key = _key(grid, scheme, precision)
    if key not in cache:
        cache[key] = lsfft_autotune(grid.handle, sigma1, e, make_opts(**kw), iters=iters)
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    ent = cache[key]
    grid.set_column_split(bool(ent["column_split"]))
    out = dict(kw)
    out["check_every"] = int(ent["check_every"])
    return out
