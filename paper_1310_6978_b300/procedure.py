"""The counting procedure of Sec. 3.4 over c-partitions, evaluated as a batch.

A good definable partition theta_1..theta_m splits every labelled model into
components; for each c-partition X (an ordered partition into consecutive
intervals, eq. (c2)) the letters fixed by the partition are killed (Sec. 3.3),
the reduced theory T_X is counted, and eq. (ltn) combines the counts:

    l_{T,n} = sum over X of  C(beta_1, alpha_1) ... C(beta_k, alpha_k) |K_X|.

Here the reduced theories are written as formula text (with ``assume``
lines) and all of them are counted in one batch (``fbg_batch_*``).  The
worked instance is Sec. 5.2: partial orders with a least element 0 and a
greatest element n-1 (two definable constants: a factor n(n-1), Sec. 3.3) whose
middle elements are split into layers of k-minimal elements; there are
2^(n-3) layer partitions (Prop. posn).
"""
from __future__ import annotations

import math
from typing import Callable, Iterable, List, Sequence

from .workloads import ANTISYMMETRIC, TRANSITIVE, Workload


def c_partition_count(n: int, m: int) -> int:
    """c_{nm} = sum_{k=1}^{m} C(m,k) C(n-1,k-1): c-partitions of an n-set into
    m possibly empty components (Prop. after eq. (kappan))."""
    return sum(math.comb(m, k) * math.comb(n - 1, k - 1) for k in range(1, m + 1))


def c_partitions(n: int, m: int) -> Iterable[tuple]:
    """All (alpha_1..alpha_m), alpha_i >= 0, summing to n: the component sizes
    of the canonical c-partitions of eq. (c2)."""
    def rec(left, parts):
        if len(parts) == m - 1:
            yield tuple(parts) + (left,)
            return
        for a in range(left + 1):
            yield from rec(left - a, parts + [a])
    if m == 0:
        if n == 0:
            yield ()
        return
    yield from rec(n, [])


def compositions(n: int) -> Iterable[tuple]:
    """Ordered partitions of n into positive parts (2^(n-1) of them, n >= 1)."""
    if n == 0:
        yield ()
        return
    for first in range(1, n + 1):
        for rest in compositions(n - first):
            yield (first,) + rest


def multinomial_weight(alphas: Sequence[int]) -> int:
    """C(beta_1, alpha_1) ... C(beta_k, alpha_k), beta_1 = sum(alpha),
    beta_{i+1} = beta_i - alpha_i (eq. (ltn))."""
    w, beta = 1, sum(alphas)
    for a in alphas:
        w *= math.comb(beta, a)
        beta -= a
    return w


def layered_bounded_poset(n: int, alphas: Sequence[int]) -> Workload:
    """T_X of Sec. 5.2 for the layers X_1..X_m of the middle elements 1..n-2
    (|X_i| = alphas[i]): 0 least and n-1 greatest (eq. (conspa)), reflexive;
    i in X_a, j in X_b with b <= a gives r(i,j) = 0 (i != j); every element of
    X_{a+1} lies above some element of X_a, so X is exactly the layer partition
    of k-minimal elements."""
    assert n >= 3 and sum(alphas) == n - 2 and all(a > 0 for a in alphas)
    layers, start = [], 1
    for a in alphas:
        layers.append(list(range(start, start + a)))
        start += a
    top = n - 1
    lines = ["var r(S,S)",
             "assume A[i:S] r(0,i)", "assume A[j:S | j>0] ~r(j,0)",
             f"assume A[i:S] r(i,{top})", f"assume A[l:S | l<{top}] ~r({top},l)",
             "assume A[i:S] r(i,i)"]
    kills = []
    for a, la in enumerate(layers):
        for b in range(a + 1):
            for i in la:
                for j in layers[b]:
                    if i != j:
                        kills.append(f"~r({i},{j})")
    for chunk in range(0, len(kills), 64):
        lines.append("assume " + " & ".join(kills[chunk:chunk + 64]))
    lines += [ANTISYMMETRIC, TRANSITIVE]
    for a in range(len(layers) - 1):
        for j in layers[a + 1]:
            lines.append(" | ".join(f"r({i},{j})" for i in layers[a]))
    free = sum(1 for i in range(1, top) for j in range(1, top) if i != j) - len(kills)
    return Workload("layered_bounded_poset", n, "\n".join(lines) + "\n", n, free)


def count_bounded_posets_by_layers(n: int, counter: Callable[[List[Workload]], List[int]]):
    """l_{T,n} for partial orders with least and greatest element on n points
    by the counting procedure: n(n-1) (definable constants, Sec. 3.3) times
    eq. (ltn) over the 2^(n-3) layer partitions.  ``counter`` counts a list of
    workloads (e.g. one GPU batch).  Returns (l, [(alphas, weight, |K_X|)])."""
    if n == 1:
        return 1, []
    if n == 2:
        return 2, []
    parts = list(compositions(n - 2))
    wls = [layered_bounded_poset(n, a) for a in parts]
    counts = counter(wls)
    detail = [(a, multinomial_weight(a), c) for a, c in zip(parts, counts)]
    return n * (n - 1) * sum(w * c for _, w, c in detail), detail


def gpu_batch_counter(workloads: List[Workload], stream=None) -> List[int]:
    """Count the workloads in one persistent batch launch."""
    from . import Batch, compile as fbg_compile
    progs = [fbg_compile(w.text, w.k) for w in workloads]
    b = Batch(progs)
    b.run(stream)
    return [int(x) for x in b.results(stream)]
