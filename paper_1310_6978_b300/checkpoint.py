"""Long counts in chunks with checkpoint and resume.

A count over 2^n assignments is a sum over the units of the count layout
(fbg_unit_vars); ``count_resumable`` evaluates the units chunk by chunk with
fbg_count_range and after every chunk writes (program key, layout, next
unit, partial count) to a JSON file.  Chunk results do not depend on each
other, so a run that stops at any point resumes from the file and ends with
the same exact count.
"""
from __future__ import annotations

import hashlib
import json
import os


def _key(prog) -> dict:
    vars_, nunits = prog.unit_vars()
    return {"formula_sha1": hashlib.sha1(prog.text.encode()).hexdigest(), "domain_k": prog.k, "n": prog.n,
            "unit_vars": vars_, "nunits": nunits}


def count_resumable(prog, path: str, chunk_units: int = 0, stream=None, max_chunks: int = 0) -> dict:
    """Count ``prog`` in chunks of units, checkpointing to ``path``.  Returns
    the state; ``state['done']`` tells whether the count is complete and
    ``state['count']`` is the (partial) count.  ``max_chunks`` > 0 stops
    after that many chunks (the file keeps the progress)."""
    key = _key(prog)
    state = {"key": key, "next_unit": 0, "count": 0, "chunks": 0, "done": False}
    if os.path.exists(path):
        with open(path) as f:
            saved = json.load(f)
        if saved.get("key") != key:
            raise ValueError(f"checkpoint {path} belongs to another program or layout")
        state = saved
    nunits = key["nunits"]
    chunk = chunk_units or max(1, nunits // 16)
    done_now = 0
    while state["next_unit"] < nunits:
        if max_chunks and done_now >= max_chunks:
            break
        end = min(nunits, state["next_unit"] + chunk)
        state["count"] += prog.count_range(state["next_unit"], end, stream)
        state["next_unit"] = end
        state["chunks"] += 1
        done_now += 1
        state["done"] = state["next_unit"] >= nunits
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(state, f)
        os.replace(tmp, path)
    state["done"] = state["next_unit"] >= nunits
    return state
