"""Independent counters -- TEST INFRASTRUCTURE ONLY.

These count finite structures directly (brute force over relations, graphs or
permutations, or classical closed forms) without any formula text, parser or
Boolean evaluation.  They pin the oracle: the number of labelled models
l_{T,n} of a theory T (Sec. 3.2) must equal the number of structures counted
here.  Nothing here is shared with the oracle or with the CUDA path.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def bell(k: int) -> int:
    """Bell numbers by the recurrence B(m+1) = sum_i C(m,i) B(i): the number
    of equivalence relations (set partitions) on k labelled points."""
    b = [1]
    for m in range(k):
        b.append(sum(math.comb(m, i) * b[i] for i in range(m + 1)))
    return b[k]


def labelled_graphs(k: int) -> int:
    """2^C(k,2): every subset of the pairs is one simple graph."""
    return 2 ** (k * (k - 1) // 2)


def _all_relations(k: int) -> np.ndarray:
    """All 2^(k^2) relations as boolean arrays [N, k, k]; bit i*k+j of the
    index is (i,j) -- used only for small k."""
    n = k * k
    idx = np.arange(1 << n, dtype=np.uint64)
    bits = ((idx[:, None] >> np.arange(n, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    return bits.reshape(-1, k, k)


def _transitive_mask(rel: np.ndarray) -> np.ndarray:
    k = rel.shape[1]
    ok = np.ones(rel.shape[0], dtype=bool)
    for i in range(k):
        for j in range(k):
            for l in range(k):
                ok &= ~(rel[:, i, j] & rel[:, j, l]) | rel[:, i, l]
    return ok


def relation_models(k: int, kind: str) -> np.ndarray:
    """Brute force over all relations on k points (k <= 4): a boolean array
    over the 2^(k^2) relations, indexed as in _all_relations, that is true
    for the relations of the given kind."""
    if k > 4:
        raise ValueError("brute force over relations only for k <= 4")
    rel = _all_relations(k)
    diag = np.stack([rel[:, i, i] for i in range(k)], axis=1)
    trans = _transitive_mask(rel)
    sym = np.ones(rel.shape[0], dtype=bool)
    anti = np.ones(rel.shape[0], dtype=bool)
    for i in range(k):
        for j in range(k):
            if i != j:
                sym &= rel[:, i, j] == rel[:, j, i]
                anti &= ~(rel[:, i, j] & rel[:, j, i])
    if kind == "poset":
        return diag.all(axis=1) & anti & trans
    if kind == "equiv":
        return diag.all(axis=1) & sym & trans
    if kind == "transitive":
        return trans
    if kind == "graph":
        return (~diag).all(axis=1) & sym
    raise ValueError(kind)


def count_relations(k: int, kind: str) -> int:
    """Brute force over all relations on k points (k <= 4)."""
    return int(np.count_nonzero(relation_models(k, kind)))


def count_posets_backtrack(k: int) -> int:
    """Partial orders on k labelled points by backtracking over the strict
    order relation, pair by pair, checking transitivity and antisymmetry of
    the pairs decided so far (the reflexive part is forced)."""
    pairs = [(i, j) for i in range(k) for j in range(k) if i != j]
    lt = [[0] * k for _ in range(k)]
    decided = [[False] * k for _ in range(k)]

    def consistent(i, j):
        # antisymmetry
        if lt[i][j] and decided[j][i] and lt[j][i]:
            return False
        # transitivity of strict order over decided pairs
        for a in range(k):
            for b in range(k):
                if a == b or not decided[a][b] or not lt[a][b]:
                    continue
                for c in range(k):
                    if c == b or c == a or not decided[b][c] or not lt[b][c]:
                        continue
                    if decided[a][c] and not lt[a][c]:
                        return False
        return True

    def rec(t):
        if t == len(pairs):
            return 1
        i, j = pairs[t]
        total = 0
        for v in (0, 1):
            lt[i][j] = v
            decided[i][j] = True
            if consistent(i, j):
                total += rec(t + 1)
            decided[i][j] = False
        lt[i][j] = 0
        return total

    return rec(0)


def triangle_free_models(k: int) -> np.ndarray:
    """Brute force over all 2^C(k,2) graphs (k <= 7), vectorised: a boolean
    array indexed by the graph whose bit t is the t-th pair a<b in
    lexicographic order, true for the triangle-free graphs."""
    pairs = [(a, b) for a in range(k) for b in range(a + 1, k)]
    m = len(pairs)
    if m > 21:
        raise ValueError("brute force only for k <= 7")
    idx = np.arange(1 << m, dtype=np.uint64)
    pos = {p: t for t, p in enumerate(pairs)}
    ok = np.ones(1 << m, dtype=bool)
    for a, b, c in itertools.combinations(range(k), 3):
        bits = np.uint64((1 << pos[(a, b)]) | (1 << pos[(b, c)]) | (1 << pos[(a, c)]))
        ok &= (idx & bits) != bits
    return ok


def count_triangle_free(k: int) -> int:
    """Brute force over all 2^C(k,2) graphs (k <= 7)."""
    return int(np.count_nonzero(triangle_free_models(k)))


def count_in_cube(models: np.ndarray, mask: int, vals: int) -> int:
    """Structures of a brute-force model array whose index has the bits of
    ``mask`` equal to those of ``vals`` (a subcube of the index space)."""
    idx = np.arange(models.shape[0], dtype=np.uint64)
    return int(np.count_nonzero(models & ((idx & np.uint64(mask)) == np.uint64(vals & mask))))


def count_automorphisms(adj_bits: str, k: int) -> int:
    """|Aut(G)| by brute force over all k! permutations of the vertices."""
    adj = [[adj_bits[i * k + j] == "1" for j in range(k)] for i in range(k)]
    total = 0
    for perm in itertools.permutations(range(k)):
        if all(adj[i][j] == adj[perm[i]][perm[j]] for i in range(k) for j in range(k)):
            total += 1
    return total


def count_transitive_backtrack(k: int) -> int:
    """Transitive relations on k labelled points (k <= 8), backtracking in C
    (oracle/counters.c) -- independent of the oracle's evaluator."""
    from . import _load
    return int(_load().counter_transitive(k))


def count_triangle_free_backtrack(k: int) -> int:
    """Triangle-free labelled graphs on k vertices (k <= 11), backtracking in C."""
    from . import _load
    return int(_load().counter_triangle_free(k))


def count_posets_c(k: int) -> int:
    """Partial orders on k labelled points (k <= 9), backtracking in C."""
    from . import _load
    return int(_load().counter_posets(k))


def count_posets_special_c(k: int) -> int:
    """Partial orders on k labelled points with an element comparable with
    every element (k <= 9), backtracking in C."""
    from . import _load
    return int(_load().counter_posets_special(k))


def count_posets_special_brute(k: int) -> int:
    """The same by brute force over all relations on k points (k <= 4)."""
    rel = _all_relations(k)
    posets = relation_models(k, "poset")
    special = np.zeros(rel.shape[0], dtype=bool)
    for a in range(k):
        ok = np.ones(rel.shape[0], dtype=bool)
        for b in range(k):
            ok &= rel[:, a, b] | rel[:, b, a]
        special |= ok
    return int(np.count_nonzero(posets & special))
