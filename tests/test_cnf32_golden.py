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
