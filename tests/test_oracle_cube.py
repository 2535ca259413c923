"""Pins for the oracle's subcube counters (no GPU).

``count_cube`` and ``count_cube_par`` count the models of a theory among the
assignments whose variables in a mask take fixed values: the definition of
Prop. 2.2 restricted to a subcube of 2^n.  The GPU parity tests check every
full-size per-unit count against ``count_cube_par``, so both are pinned here
against brute force over structures (oracle/counters.py, no formula text),
against each other, against the whole-range count (empty mask) and a single
evaluation (full mask), and at the loop bound (63 and 64 free variables).
"""
import numpy as np
import pytest

import oracle
from oracle import counters as C
from paper_1310_6978_b300 import workloads as W


def _random_cubes(n, rng, count):
    out = [(0, 0), ((1 << n) - 1, int(rng.integers(0, 1 << n)))]
    for _ in range(count):
        mask = int(rng.integers(0, 1 << n))
        out.append((mask, int(rng.integers(0, 1 << n)) & mask))
    return out


@pytest.mark.parametrize("kind,k", [("poset", 4), ("equiv", 4), ("transitive", 3), ("graph", 4)])
def test_cube_counts_equal_brute_force_over_relations(kind, k):
    wl = {"poset": W.posets, "equiv": W.equivalences, "transitive": W.transitive, "graph": W.graphs}[kind](k)
    th = oracle.Theory(wl.text, k)
    models = C.relation_models(k, kind)
    rng = np.random.default_rng(k * 7 + len(kind))
    for mask, vals in _random_cubes(th.n, rng, 12):
        want = C.count_in_cube(models, mask, vals)
        assert th.count_cube(mask, vals) == want, (mask, vals)
        assert th.count_cube_par(mask, vals, 4) == want, (mask, vals)


@pytest.mark.parametrize("k", [5, 6])
def test_cube_counts_equal_brute_force_over_graphs(k):
    th = oracle.Theory(W.triangle_free(k).text, k)
    models = C.triangle_free_models(k)
    rng = np.random.default_rng(k)
    for mask, vals in _random_cubes(th.n, rng, 10):
        want = C.count_in_cube(models, mask, vals)
        assert th.count_cube(mask, vals) == th.count_cube_par(mask, vals) == want, (mask, vals)


def test_cube_counters_agree_on_random_cnf():
    wl = W.cnf3(18, 4)
    th = oracle.Theory(wl.text, wl.k)
    rng = np.random.default_rng(3)
    for mask, vals in _random_cubes(th.n, rng, 20):
        a = th.count_cube(mask, vals)
        assert th.count_cube_par(mask, vals, 1) == a
        assert th.count_cube_par(mask, vals, 3) == a
        assert th.count_cube_par(mask, vals) == a
        if bin(mask).count("1") >= 8:   # few free variables: enumerate the cube point by point
            free = [i for i in range(th.n) if not (mask >> i) & 1]
            pts = [(vals & mask) | sum(((t >> b) & 1) << v for b, v in enumerate(free)) for t in range(1 << len(free))]
            assert a == sum(th.eval(j) for j in pts)


def test_empty_and_full_masks():
    wl = W.posets(4)
    th = oracle.Theory(wl.text, 4)
    assert th.count_cube(0, 0) == th.count_cube_par(0, 0) == th.count() == 219
    full = (1 << th.n) - 1
    for j in (0, 1, 0b1000010000100001, full):
        assert th.count_cube(full, j) == th.count_cube_par(full, j) == th.eval(j)


def test_loop_bound_at_63_and_64_free_variables():
    # both counters share one loop bound: 2^nf points for nf <= 63 (2^63 fits
    # an unsigned 64-bit count), and a refusal at nf = 64
    assert oracle.cube_size(0) == 1
    assert oracle.cube_size(1) == 2
    assert oracle.cube_size(62) == 1 << 62
    assert oracle.cube_size(63) == 1 << 63
    assert oracle.cube_size(64) is None
    th = oracle.Theory("var x(S)\nx(0) | ~x(0)\n", 64)
    assert th.n == 64
    with pytest.raises(ValueError):
        th.count_cube(0, 0)
    with pytest.raises(ValueError):
        th.count_cube_par(0, 0)
    # 63 fixed: one free variable, the tautology holds on both points
    assert th.count_cube(((1 << 64) - 1) ^ 1, 0) == th.count_cube_par(((1 << 64) - 1) ^ 2, 0) == 2
