"""Checks of GPU results against the oracle at sizes where the oracle cannot
evaluate every assignment in a test's time (test infrastructure).

* Counts: below ``full_max_n`` letters the oracle counts all 2^n points.
  Above it the library's interpreter counts the same text per unit (at most
  2^16 units, so at least 2^(n-16) assignments each); the per-unit counts
  must add up to the result under test, and sampled units (plus the first and
  the last) must equal the oracle's count over the same subcube (the
  definition of Prop. 2.2 restricted to it).
* Model lists (ascending j, the first ``cap`` models): below ``full_max_n``
  the oracle's own list; above it every sampled listed model satisfies the
  theory, the list is strictly ascending, its length is min(cap, total), and
  sampled gaps between consecutive models (and the range before the first)
  hold no model of the oracle.
"""
from __future__ import annotations

import numpy as np

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L


def _theory(wl, cache):
    key = (wl.text, wl.k)
    if cache is None:
        return oracle.Theory(wl.text, wl.k)
    if key not in cache:
        cache[key] = oracle.Theory(wl.text, wl.k)
    return cache[key]


def check_count(wl, count: int, rng, *, full_max_n: int = 22, unit_points: int = 18, samples: int = 2,
                cache: dict | None = None) -> str:
    """Assert that ``count`` is the number of models of ``wl`` (a workload);
    returns how it was checked ("full" or "units")."""
    import torch
    th = _theory(wl, cache)
    assert th.n == wl.n
    if wl.n <= full_max_n:
        want = th.count_par(0, 1 << wl.n) if wl.n > 16 else th.count()
        assert count == want, (wl, count, want)
        return "full"
    p = F.compile(wl.text, wl.k).set_option(L.OPT_ENGINE, L.ENGINE_INTERP)
    p.set_option(L.OPT_UNIT_BITS, min(16, max(0, wl.n - unit_points)))
    vars_, nunits = p.unit_vars()
    dev = torch.zeros(nunits, dtype=torch.int64, device="cuda")
    p.count_units(dev)
    uc = np.array(F.read_counts(dev), dtype=object)
    assert sum(int(x) for x in uc) == count, (wl, count)
    mask = sum(1 << v for v in vars_)
    picks = {0, nunits - 1} | {int(u) for u in rng.integers(0, nunits, samples)}
    for u in sorted(picks):
        vals = sum(((u >> b) & 1) << v for b, v in enumerate(vars_))
        assert int(uc[u]) == th.count_cube_par(mask, vals), (wl, "unit", u)
    return "units"


def check_models(wl, models, total: int, cap: int, rng, *, full_max_n: int = 22, samples: int = 2000,
                 gaps: int = 24, max_gap_bits: int = 22, cache: dict | None = None) -> str:
    """Assert that ``models`` (ints) is the ascending list of the first
    ``cap`` models of ``wl`` whose exact number is ``total``."""
    th = _theory(wl, cache)
    models = np.asarray([int(m) for m in models], dtype=np.uint64)
    assert len(models) == min(cap, total), (wl, len(models), cap, total)
    if wl.n <= full_max_n:
        want, want_total = th.models(cap)
        assert want_total == total and np.array_equal(want, models), wl
        return "full"
    if len(models) == 0:
        return "empty"
    assert np.all(np.diff(models.astype(np.float64)) > 0) and np.all(models[1:] > models[:-1]), wl
    assert int(models[-1]) < (1 << wl.n)
    idx = rng.choice(len(models), min(samples, len(models)), replace=False)
    for i in idx:
        assert th.eval(int(models[i])) == 1, (wl, int(models[i]))
    # no model is missing between listed ones (or before the first)
    lim = 1 << max_gap_bits
    if int(models[0]) <= lim:
        assert th.count_par(0, int(models[0])) == 0, (wl, "before first")
    cand = [i for i in range(len(models) - 1) if int(models[i + 1]) - int(models[i]) - 1 <= lim]
    for i in (rng.choice(cand, min(gaps, len(cand)), replace=False) if cand else []):
        lo, hi = int(models[i]) + 1, int(models[i + 1])
        assert th.count_par(lo, hi) == 0, (wl, "gap", lo, hi)
    return "sampled"
