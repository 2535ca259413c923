"""The stored full-size 3-CNF tables (tests/golden/cnf32_seed*.txt, written
by the oracle over all 2^32 assignments) pinned by a procedure that shares
nothing with the oracle: a small DPLL satisfiability search over the clause
list.  Seed 1 (the benchmark's formula) is unsatisfiable, so its stored
count must be 0 and its stored hash that of 2^26 zero words; seed 2 is
satisfiable, so the oracle must accept the assignment DPLL finds and the
stored count must be positive."""
import hashlib
import os
import re

import oracle
from paper_1310_6978_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    return {k: v for k, v in rows}


def _clauses(text):
    out = []
    for ln in text.splitlines()[1:]:
        lits = []
        for t in ln.split("|"):
            t = t.strip()
            v = int(re.search(r"\((\d+)\)", t).group(1))
            lits.append(-(v + 1) if t.startswith("~") else v + 1)
        out.append(lits)
    return out


def _dpll(cl, assign):
    """A satisfying partial assignment {var: bool} (1-based vars), or None."""
    changed = True
    while changed:
        changed = False
        for c in cl:
            free, sat = [], False
            for lit in c:
                v = assign.get(abs(lit))
                if v is None:
                    free.append(lit)
                elif v == (lit > 0):
                    sat = True
                    break
            if sat:
                continue
            if not free:
                return None
            if len(free) == 1:
                assign[abs(free[0])] = free[0] > 0
                changed = True
    for c in cl:
        for lit in c:
            if abs(lit) not in assign:
                for val in (lit > 0, lit < 0):
                    a = dict(assign)
                    a[abs(lit)] = val
                    r = _dpll(cl, a)
                    if r is not None:
                        return r
                return None
    return assign


def test_seed1_is_unsatisfiable_and_its_table_is_zero():
    assert W.CNF32.text == W.cnf3(32, 1).text
    assert _dpll(_clauses(W.CNF32.text), {}) is None
    g = _golden("cnf32_seed1.txt")
    assert int(g["count"]) == 0
    h = hashlib.sha256()
    zeros = bytes(1 << 20)
    for _ in range(512):          # 2^26 words of 8 bytes = 512 MiB
        h.update(zeros)
    assert g["sha256"] == h.hexdigest()


def test_seed2_model_found_by_dpll_is_an_oracle_model():
    wl = W.cnf3(32, 2)
    a = _dpll(_clauses(wl.text), {})
    assert a is not None
    j = sum(1 << (v - 1) for v, val in a.items() if val)   # unassigned letters: 0
    assert oracle.Theory(wl.text, wl.k).eval(j) == 1
    assert int(_golden("cnf32_seed2.txt")["count"]) >= 1


def _count_models(cl, nvars):
    """Exact model count by DPLL branching with unit propagation: a branch
    whose clauses are all satisfied counts 2^(unassigned letters).  Shares
    nothing with the oracle (no formula text, no evaluation per point)."""
    def rec(clauses, assigned):
        changed = True
        clauses = [list(c) for c in clauses]
        assigned = dict(assigned)
        while changed:
            changed = False
            nxt = []
            for c in clauses:
                free, sat = [], False
                for lit in c:
                    v = assigned.get(abs(lit))
                    if v is None:
                        free.append(lit)
                    elif v == (lit > 0):
                        sat = True
                        break
                if sat:
                    continue
                if not free:
                    return 0
                if len(free) == 1:
                    assigned[abs(free[0])] = free[0] > 0
                    changed = True
                nxt.append(free)
            clauses = nxt
        if not clauses:
            return 1 << (nvars - len(assigned))
        # branch on the most frequent free letter
        freq = {}
        for c in clauses:
            for lit in c:
                freq[abs(lit)] = freq.get(abs(lit), 0) + 1
        v = max(freq, key=lambda x: (freq[x], -x))
        return rec(clauses, {**assigned, v: True}) + rec(clauses, {**assigned, v: False})
    return rec(cl, {})


def test_dpll_counter_on_small_formulas_matches_brute_force():
    import itertools
    for seed in (1, 2, 3):
        wl = W.cnf3(12, seed, 2.0)
        cl = _clauses(wl.text)
        brute = sum(all(any((bits[abs(l) - 1] == 1) == (l > 0) for l in c) for c in cl)
                    for bits in itertools.product((0, 1), repeat=12))
        assert _count_models(cl, 12) == brute


def test_dense_ratio2_seed3_count_equals_dpll_count():
    # the dense table of the benchmark (ratio 2, m = 64, seed 3): the oracle's
    # stored count equals an exact DPLL model count of the clause list
    wl = W.cnf3(32, 3, 2.0)
    cl = _clauses(wl.text)
    assert len(cl) == 64
    assert int(_golden("cnf32_r2_seed3.txt")["count"]) == _count_models(cl, 32) == 624090
