"""The counting procedure of Sec. 3.4 over c-partitions, evaluated as a batch.

A good definable partition theta_1..theta_m splits every labelled model into
components; for each c-partition X (an ordered partition into consecutive
intervals, eq. (c2)) the letters fixed by the partition are killed (Sec. 3.3),
the reduced theory T_X is counted, and eq. (ltn) combines the counts:

    l_{T,n} = sum over X of  C(beta_1, alpha_1) ... C(beta_k, alpha_k) |K_X|.

Here the reduced theories are written as formula text (with ``assume``
lines) and all of them are counted in one batch (``fbg_batch_*``).
``count_by_partition`` runs the procedure for any theory given its good
definable partition (the formulas theta_k and the literals S_kl); two
instances are provided: the layers of Sec. 5.2 (partial orders with a least
element 0 and a greatest element n-1, two definable constants: a factor
n(n-1), Sec. 3.3, middle elements split into layers of k-minimal elements,
2^(n-3) layer partitions, Prop. posn) and the minimal / non-minimal split of
partial orders with a special element (the SO.txt script of Sec. 4.2).
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


# -- the procedure for any theory with a good definable partition ------------

# S_kl(x, y) of a good definable partition (Sec. 3.4): for x in X_k, y in X_l,
# k <= l, the theory proves one of these literals; each kills one letter.
S_FORMS = ("R(x,y)", "R(y,x)", "~R(x,y)", "~R(y,x)")


def partition_kills(comps: Sequence[Sequence[int]], S: dict, rel: str = "r", distinct: bool = True) -> List[str]:
    """Step 3 (killing variables): for every pair of components k <= l with a
    form S[(k, l)] and every x in X_k, y in X_l (x != y when ``distinct``,
    the reading for reflexive relations), the literal that S_kl fixes, as
    formula text ("r(2,5)" or "~r(5,2)").  Components are numbered from 1."""
    lits = {}
    for k in range(1, len(comps) + 1):
        for l in range(k, len(comps) + 1):
            form = S.get((k, l))
            if form is None:
                continue
            if form not in S_FORMS:
                raise ValueError(f"S[{k},{l}] must be one of {S_FORMS}")
            neg = form.startswith("~")
            swap = "R(y,x)" in form
            for x in comps[k - 1]:
                for y in comps[l - 1]:
                    if distinct and x == y:
                        continue
                    a, b = (y, x) if swap else (x, y)
                    lit = f"{rel}({a},{b})"
                    want = f"~{lit}" if neg else lit
                    if lits.get(lit, want) != want:
                        raise ValueError(f"S fixes {lit} both ways: not a good partition")
                    lits[lit] = want
    return list(lits.values())


def canonical_components(alphas: Sequence[int]) -> List[List[int]]:
    """The canonical arrangement of eq. (c2): X_1 = {0..alpha_1-1}, X_2 the
    next alpha_2 elements, and so on."""
    comps, start = [], 0
    for a in alphas:
        comps.append(list(range(start, start + a)))
        start += a
    return comps


def partition_theory(base_text: str, alphas: Sequence[int], theta: Callable[[int, int], str], S: dict,
                     rel: str = "r", distinct: bool = True) -> str:
    """T_X (step 4): the theory text, the letters killed by S for the
    c-partition X of sizes ``alphas`` (as ``assume`` lines), and theta_k(x)
    for every x in X_k (so that Delta defines exactly X in every model of
    T_X).  ``theta(k, x)`` returns the formula text of theta_k at the
    element x."""
    comps = canonical_components(alphas)
    lines = [base_text.rstrip("\n")]
    kills = partition_kills(comps, S, rel, distinct)
    for c in range(0, len(kills), 64):
        lines.append("assume " + " & ".join(kills[c:c + 64]))
    for k, comp in enumerate(comps, start=1):
        for x in comp:
            lines.append(theta(k, x))
    return "\n".join(lines) + "\n"


def count_by_partition(base_text: str, n: int, m: int, theta: Callable[[int, int], str], S: dict,
                       counter: Callable[[List[Workload]], List[int]], rel: str = "r", distinct: bool = True,
                       factor: int = 1):
    """l_{T,n} by the counting procedure of Sec. 3.4 (steps 1-8): every
    c-partition X = (X_1..X_m) of I_n in the arrangement (c2) (component sizes
    alpha_i >= 0, c_{nm} of them), its reduced theory T_X counted by
    ``counter`` (all of them in one call, e.g. one GPU batch), and eq. (ltn):
    l = factor * sum_X C(beta_1, alpha_1)...C(beta_m, alpha_m) |K_X|.
    ``factor`` carries the n(n-1)..(n-k+1) of k definable constants killed
    in ``base_text`` (Sec. 3.3).  Returns (l, [(alphas, weight, |K_X|)])."""
    parts = list(c_partitions(n, m))
    wls = [Workload("partition", n, partition_theory(base_text, a, theta, S, rel, distinct), n, -1) for a in parts]
    counts = counter(wls)
    detail = [(a, multinomial_weight(a), c) for a, c in zip(parts, counts)]
    return factor * sum(w * c for _, w, c in detail), detail


# Posets with a special element (the SO.txt script of Sec. 4.2) and the
# partition into minimal and non-minimal elements: theta_1(x) says nothing
# lies strictly below x, theta_2(x) that something does; S_11 = ~R(x,y) (two
# minimal elements are incomparable), S_12 = ~R(y,x) (nothing lies strictly
# below a minimal element); no literal holds between two non-minimal ones.
def minimal_theta(k: int, x: int, rel: str = "r") -> str:
    if k == 1:
        return f"A[y:S | y != {x}] ~{rel}(y,{x})"
    return f"E[y:S | y != {x}] {rel}(y,{x})"


MINIMAL_S = {(1, 1): "~R(x,y)", (1, 2): "~R(y,x)"}


def gpu_batch_counter(workloads: List[Workload], stream=None) -> List[int]:
    """Count the workloads in one persistent batch launch."""
    from . import Batch, compile as fbg_compile
    progs = [fbg_compile(w.text, w.k) for w in workloads]
    b = Batch(progs)
    b.run(stream)
    return [int(x) for x in b.results(stream)]
