"""Unlabelled models: kappa_{T,n} of Sec. 3.2 from the labelled model list.

The labelled models of T on I_n (the ascending model list of
fbg_enumerate_models) are grouped into isomorphism classes: a relabelling
alpha of the domain permutes the letters (R(i,j) -> R(alpha(i), alpha(j))),
so each class is the orbit of any of its members under all n! relabellings.
Orbits are generated one at a time from the first model not yet covered, all
n! images at once with numpy.  By the labelling theorem of Sec. 3.2 an orbit
has n!/|Aut(A)| elements, so the Frobenius-Burnside identity
l_n = sum_A n!/|Aut(A)| holds by construction and is reported as a check.
"""
from __future__ import annotations

import itertools
import math
import re

import numpy as np


def letter_permutations(prog, k: int) -> np.ndarray:
    """For every relabelling of range(k), the letter index each letter maps
    to: array [k!, n].  Letters are named f(i,..) (fbg_var_name); a family
    declared with increasing positions (S<S) is looked up in sorted order."""
    names = [prog.var_name(i) for i in range(prog.n)]
    index = {nm: i for i, nm in enumerate(names)}
    parsed = []
    for nm in names:
        m = re.fullmatch(r"([A-Za-z_][A-Za-z0-9_]*)(?:\(([0-9,]*)\))?", nm)
        if not m:
            raise ValueError(f"cannot relabel letter {nm}")
        args = tuple(int(x) for x in m.group(2).split(",")) if m.group(2) else ()
        parsed.append((m.group(1), args))
    perms = list(itertools.permutations(range(k)))
    table = np.empty((len(perms), len(names)), dtype=np.int64)
    for pi, perm in enumerate(perms):
        for li, (fam, args) in enumerate(parsed):
            img = tuple(perm[a] for a in args)
            key = f"{fam}({','.join(map(str, img))})" if args else fam
            if key not in index:
                key = f"{fam}({','.join(map(str, sorted(img)))})"
            if key not in index:
                raise ValueError(f"relabelling leaves the letter set: {key}")
            table[pi, li] = index[key]
    return table


def orbits(models: np.ndarray, table: np.ndarray):
    """Isomorphism classes of the models (uint64 assignment integers, bit i =
    letter i) under the letter permutations in ``table``: list of orbit sizes
    and one representative (the smallest member) per class."""
    models = np.unique(np.asarray(models, dtype=np.uint64))
    n = table.shape[1]
    covered = np.zeros(models.shape[0], dtype=bool)
    bits_idx = np.arange(n, dtype=np.uint64)
    sizes, reps = [], []
    for start in range(models.shape[0]):
        if covered[start]:
            continue
        m = models[start]
        bits = ((m >> bits_idx) & np.uint64(1)).astype(np.uint64)          # [n]
        # image of m under relabelling p: bit table[p, i] of the image = bit i of m
        images = np.zeros(table.shape[0], dtype=np.uint64)
        for i in range(n):
            images |= bits[i] << table[:, i].astype(np.uint64)
        orbit = np.unique(images)
        pos = np.searchsorted(models, orbit)
        ok = (pos < models.shape[0])
        ok[ok] = models[pos[ok]] == orbit[ok]
        if not ok.all():
            raise ValueError("the model list is not closed under relabelling (incomplete list?)")
        covered[pos] = True
        sizes.append(int(orbit.shape[0]))
        reps.append(int(orbit[0]))
    return sizes, reps


def unlabelled_count(prog, k: int, stream=None, cap: int = 1 << 24) -> dict:
    """kappa_{T,k} and the Frobenius-Burnside check for a compiled theory
    over a k-element domain (no killed letters): enumerates every model on the
    GPU, then counts the orbits."""
    import torch
    buf = torch.empty(cap, dtype=torch.int64, device="cuda")
    total, written = prog.enumerate_models(buf, cap, stream)
    if written < total:
        raise ValueError(f"{total} models exceed the capacity {cap}")
    models = buf[:written].cpu().numpy().view(np.uint64)
    table = letter_permutations(prog, k)
    sizes, reps = orbits(models, table)
    fact = math.factorial(k)
    auts = [fact // s for s in sizes]
    return {"labelled": int(total), "unlabelled": len(sizes),
            "burnside_sum": sum(fact // a for a in auts),
            "automorphism_group_orders": auts, "representatives": reps}
