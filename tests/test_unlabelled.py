"""Unlabelled counts (Sec. 3.2) on the CPU from oracle model lists: orbit
counting against partition numbers (equivalence relations), graph
isomorphism classes computed by networkx, and the Frobenius-Burnside
identity l_n = sum n!/|Aut(A)|."""
import math

import networkx as nx
import numpy as np
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import unlabelled as U
from paper_1310_6978_b300 import workloads as W


def partitions(k):
    """Partition numbers by Euler's recurrence over generalised pentagonal numbers."""
    p = [1] + [0] * k
    for m in range(1, k + 1):
        s, j = 0, 1
        while True:
            g1, g2 = j * (3 * j - 1) // 2, j * (3 * j + 1) // 2
            if g1 > m:
                break
            sign = 1 if j % 2 else -1
            s += sign * p[m - g1]
            if g2 <= m:
                s += sign * p[m - g2]
            j += 1
        p[m] = s
    return p[k]


def orbits_of(wl):
    th = oracle.Theory(wl.text, wl.k)
    models, total = th.models(1 << 20)
    assert len(models) == total
    prog = F.compile(wl.text, wl.k)
    sizes, reps = U.orbits(models, U.letter_permutations(prog, wl.k))
    assert sum(sizes) == total                                     # l_n = sum n!/|Aut|
    assert all(math.factorial(wl.k) % s == 0 for s in sizes)        # orbit sizes divide n!
    return sizes, reps


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_equivalence_classes_are_partitions(k):
    sizes, _ = orbits_of(W.equivalences(k))
    assert len(sizes) == partitions(k)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_graph_classes_match_networkx(k):
    sizes, reps = orbits_of(W.graphs(k))
    th = oracle.Theory(W.graphs(k).text, k)
    models, _ = th.models(1 << 20)
    classes = []
    for m in models:
        m = int(m)
        g = nx.Graph()
        g.add_nodes_from(range(k))
        g.add_edges_from((i, j) for i in range(k) for j in range(i + 1, k) if (m >> (i * k + j)) & 1)
        if not any(nx.is_isomorphic(g, h) for h in classes):
            classes.append(g)
    assert len(sizes) == len(classes)


def test_triangle_free_pair_family_and_small_posets():
    sizes, _ = orbits_of(W.triangle_free(4))
    th = oracle.Theory(W.triangle_free(4).text, 4)
    models, _ = th.models(1 << 10)
    pairs = [(a, b) for a in range(4) for b in range(a + 1, 4)]
    classes = []
    for m in models:
        g = nx.Graph()
        g.add_nodes_from(range(4))
        g.add_edges_from(p for t, p in enumerate(pairs) if (int(m) >> t) & 1)
        if not any(nx.is_isomorphic(g, h) for h in classes):
            classes.append(g)
    assert len(sizes) == len(classes)
    psizes, _ = orbits_of(W.posets(4))
    assert sum(psizes) == 219


def test_incomplete_list_is_rejected():
    prog = F.compile(W.equivalences(3).text, 3)
    th = oracle.Theory(W.equivalences(3).text, 3)
    models, _ = th.models(100)
    with pytest.raises(ValueError):
        # drop a member of the 3-element orbit of one-pair equivalences
        U.orbits(np.delete(models, 1), U.letter_permutations(prog, 3))
