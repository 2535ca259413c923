"""Cache of kernel shapes chosen by the autotuner (fbg_autotune).

Shapes are keyed by the formula text, domain size and mode and stored as
JSON.  ``tuned_shapes.json`` beside this file holds the shapes tuned on a
B300 for the benchmark workloads; other programs keep the default shape
unless ``ensure`` is asked to tune them.
"""
from __future__ import annotations

import hashlib
import json
import os

DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_shapes.json")


def key(text: str, k: int, mode: int) -> str:
    return f"{hashlib.sha1(text.encode()).hexdigest()[:16]}:k{k}:m{mode}"


def load(path: str = DEFAULT_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(cache: dict, path: str) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def ensure(prog, mode: int = 0, cache: dict | None = None, tune: bool = False, stream=None, reps: int = 3,
           refine: bool = False):
    """Apply the cached shape of ``prog`` (a Program) if there is one; else,
    with ``tune``, run the autotuner and record its choice in ``cache``.  With
    ``refine`` the autotuner also runs on a cached shape, starting from it.  Returns the shape applied (or None)."""
    cache = load() if cache is None else cache
    kk = key(prog.text, prog.k, mode)
    if kk in cache and not refine:
        prog.apply_shape(cache[kk])
        return cache[kk]
    if kk in cache:
        # the search starts from (and times) the cached shape, so its result
        # is at least as fast on this GPU
        prog.apply_shape(cache[kk])
        cache[kk] = prog.autotune(mode, reps, stream)
        return cache[kk]
    if not tune:
        return None
    shape = prog.autotune(mode, reps, stream)
    cache[kk] = shape
    return shape
