"""Function symbols (Sec. 3.1: F(a..) = b coded by the letter p_{Fa..b}).

The oracle is pinned against brute force over operation tables written
without any formula text, against closed forms (injective maps on a finite
set are the k! permutations, a constant symbol has k values) and against the
known numbers of semigroups up to isomorphism."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1310_6978_b300 import workloads as W


def tables(k, cells):
    return itertools.product(range(k), repeat=cells)


def brute_semigroups(k):
    n = 0
    for t in tables(k, k * k):
        m = lambda a, b: t[a * k + b]
        n += all(m(m(x, y), z) == m(x, m(y, z)) for x in range(k) for y in range(k) for z in range(k))
    return n


def is_latin(t, k):
    rows = all(len({t[a * k + b] for b in range(k)}) == k for a in range(k))
    cols = all(len({t[a * k + b] for a in range(k)}) == k for b in range(k))
    return rows and cols


@pytest.mark.parametrize("k,expected", [(1, 1), (2, 8), (3, 113)])
def test_semigroups_brute_force(k, expected):
    assert brute_semigroups(k) == expected
    assert oracle.Theory(W.semigroups(k).text, k).count() == expected


def test_latin_squares_brute_force():
    k = 3
    all_latin = [t for t in tables(k, k * k) if is_latin(t, k)]
    assert len(all_latin) == 12
    assert oracle.Theory(W.latin_squares(3).text, 3).count() == 12
    row = [t for t in all_latin if t[:k] == tuple(range(k))]
    th = oracle.Theory(W.latin_squares(3, first_row=True).text, 3)
    assert th.n == 27 - 9 and th.count() == len(row) == 2
    # order 4: first row and column fixed (reduced squares), 4 of them
    k = 4
    cnt = 0
    for t in tables(k, (k - 1) * (k - 1)):
        full = list(range(k))
        for i in range(1, k):
            full += [i] + [t[(i - 1) * (k - 1) + (j - 1)] for j in range(1, k)]
        cnt += is_latin(full, k)
    th = oracle.Theory(W.reduced_latin_squares(4).text, 4)
    assert th.n == W.reduced_latin_squares(4).n == 21
    assert th.count() == cnt == 4


def test_groups_small():
    # labelled groups on k points: sum over iso types of k!/|Aut|
    assert oracle.Theory(W.groups(2).text, 2).count() == 2          # Z2: 2!/1
    assert oracle.Theory(W.groups(3).text, 3).count() == 3          # Z3: 3!/2
    assert oracle.Theory(W.groups_identity0(3).text, 3).count() == 1


def test_model_decodes_to_the_operation_table():
    k = 2
    th = oracle.Theory(W.semigroups(k).text, k)
    models, total = th.models(1 << 8)
    got = set()
    for j in models:
        j = int(j)
        t = []
        for a in range(k):
            for b in range(k):
                vals = [u for u in range(k) if (j >> ((a * k + b) * k + u)) & 1]
                assert len(vals) == 1                                  # a function
                t.append(vals[0])
        got.add(tuple(t))
    want = {t for t in tables(k, k * k)
            if all(t[t[x * k + y] * k + z] == t[x * k + t[y * k + z]] for x in range(k) for y in range(k) for z in range(k))}
    assert got == want


def test_constant_symbol_and_equations():
    assert oracle.Theory("fun c\n", 3).count() == 3                    # exactly one value
    assert oracle.Theory("fun c\nc = 1\n", 3).count() == 1
    th = oracle.Theory("fun c\nc = 1\n", 3)
    assert [int(x) for x in th.models(8)[0]] == [0b010]
    # injective maps on a k-set are its k! permutations
    for k in (2, 3, 4):
        th = oracle.Theory("fun f(S)\nA[x,y:S] (x != y -> f(x) != f(y))\n", k)
        assert th.count() == math.factorial(k)
    # a label is not confused with an equation whose left side is a symbol
    assert oracle.Theory("fun c\ne1 = c = 2\n", 3).count() == 1


def test_function_terms_inside_relation_atoms():
    k = 3
    th = oracle.Theory("var r(S)\nfun f(S)\nA[x:S] r(f(x))\n", k)
    want = sum(2 ** (k - len(set(t))) for t in tables(k, k))
    assert th.count() == want
    th = oracle.Theory("var r(S,S)\nfun f(S)\nA[x:S] r(x, f(f(x)))\n", 2)
    want = 0
    for t in tables(2, 2):
        for bits in range(16):
            want += all((bits >> (x * 2 + t[t[x]])) & 1 for x in range(2))
    assert th.count() == want


def test_assume_on_a_function_value_kills_its_row():
    th = oracle.Theory("fun m(S,S)\nassume m(0,0) = 1\n", 3)
    assert th.n == 27 - 3 and th.count() == 3 ** 8
    th = oracle.Theory("fun m(S,S)\nassume ~(m(0,0) = 1)\n", 3)
    assert th.n == 26 and th.count() == 2 * 3 ** 8
    with pytest.raises(oracle.OracleError):
        oracle.Theory("fun m(S,S)\nassume m(m(0,0),0) = 1\n", 3)
    with pytest.raises(oracle.OracleError):
        oracle.Theory("var e(S<S)\nfun f(S)\nA[x:S] e(x, f(x))\n", 3)
    with pytest.raises(oracle.OracleError):
        oracle.Theory("fun m(S,S)\nm(0,3) = 0\n", 3)



def test_unlabelled_semigroups():
    import paper_1310_6978_b300 as F
    from paper_1310_6978_b300 import unlabelled as U
    for k, labelled, unlabelled in ((2, 8, 5), (3, 113, 24)):
        wl = W.semigroups(k)
        models, total = oracle.Theory(wl.text, k).models(1 << 10)
        prog = F.compile(wl.text, k)
        sizes, _ = U.orbits(models, U.letter_permutations(prog, k))
        assert total == labelled and sum(sizes) == labelled and len(sizes) == unlabelled
