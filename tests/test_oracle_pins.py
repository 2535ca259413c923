"""Pins for the CPU oracle (no GPU).

The oracle is checked against things fixed outside itself: the generator
matrix printed in Sec. 2.2, the independence of free generators (every
minterm is non-zero, Sec. 2.2), the Boolean system BAequ4 of Sec. 5.1 solved
here by plain integer arithmetic, closed forms (Bell numbers, 2^C(k,2)
graphs, 19/219/4231 labelled posets), brute force over structures
(oracle/counters.py) and identities every count satisfies.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import counters as C
from paper_1310_6978_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def bits_string(words, n):
    return "".join(str((int(words[j >> 6]) >> (j & 63)) & 1) for j in range(1 << n))


def test_generators_match_matrix_of_sec_2_2():
    rows = {}
    for line in open(os.path.join(GOLDEN, "generators_n3.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, bits = line.split()
        rows[name] = bits
    n = 3
    for m in range(1, n + 1):
        # b_m is the (m)-th most significant digit of j: our x_{n-m}
        th = oracle.Theory(W.single_var(n, n - m).text)
        assert bits_string(th.table(), n) == rows[f"b{m}"]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 7])
def test_minterms_are_single_bits(n):
    # independence: b_1^a1 & ... & b_n^an != 0, and for these generators
    # each minterm is exactly the one position alpha
    for alpha in range(1 << n):
        th = oracle.Theory(W.minterm(n, alpha).text)
        t = th.table()
        ones = [j for j in range(1 << n) if (int(t[j >> 6]) >> (j & 63)) & 1]
        assert ones == [alpha]


def test_table_tail_is_zero_below_six_vars():
    th = oracle.Theory("var a, b\na | ~a\n")
    t = th.table()
    assert t.shape == (1,) and int(t[0]) == 0xF


def test_baequ4_solutions_by_arithmetic():
    text = "var x, y, z, u\n" + open(os.path.join(GOLDEN, "baequ4.txt")).read()
    th = oracle.Theory(text)
    models, total = th.models(16)
    expected = []
    for j in range(16):
        x, y, z, u = (j >> 0) & 1, (j >> 1) & 1, (j >> 2) & 1, (j >> 3) & 1
        if (x + y + (1 - z) + u) % 2 == 1 and (x | (y & z)) == u:
            expected.append(j)
    assert list(models) == expected
    assert total == 3
    assert sorted(((j & 1), (j >> 1) & 1, (j >> 2) & 1, (j >> 3) & 1) for j in expected) == \
        [(0, 0, 0, 0), (1, 0, 0, 1), (1, 1, 1, 1)]


@pytest.mark.parametrize("op,py", [
    ("&", lambda a, b: a & b), ("|", lambda a, b: a | b), ("^", lambda a, b: a ^ b),
    ("->", lambda a, b: (1 - a) | b), ("<->", lambda a, b: 1 - (a ^ b)),
])
def test_binary_operators(op, py):
    th = oracle.Theory(f"var a, b\na {op} b\n")
    assert [th.eval(j) for j in range(4)] == [py(j & 1, j >> 1) for j in range(4)]


def test_precedence_python_order():
    # ~ > & > ^ > | ; -> right associative below | ; <-> lowest
    th = oracle.Theory("var a, b, c\na | b & c ^ ~a\n")
    for j in range(8):
        a, b, c = j & 1, (j >> 1) & 1, (j >> 2) & 1
        assert th.eval(j) == (a | ((b & c) ^ (1 - a)))
    th = oracle.Theory("var a, b, c\na -> b -> c\n")
    for j in range(8):
        a, b, c = j & 1, (j >> 1) & 1, (j >> 2) & 1
        assert th.eval(j) == ((1 - a) | ((1 - b) | c))
    th = oracle.Theory("var a, b, c\na <-> b | c\n")
    for j in range(8):
        a, b, c = j & 1, (j >> 1) & 1, (j >> 2) & 1
        assert th.eval(j) == int(a == (b | c))


def test_variable_numbering_lexicographic():
    # r(i,j) has id i*k+j; e(a<b) ranks pairs lexicographically
    th = oracle.Theory("var r(S,S)\nr(1,2)\n", 3)
    assert th.n == 9
    assert th.eval(1 << (1 * 3 + 2)) == 1 and th.eval(1 << (2 * 3 + 1)) == 0
    th = oracle.Theory("var e(S<S)\ne(1,3)\n", 4)
    pairs = [(a, b) for a in range(4) for b in range(a + 1, 4)]
    assert th.n == 6 and th.eval(1 << pairs.index((1, 3))) == 1


def test_quantifier_sets_and_guards():
    k = 4
    th_s2 = oracle.Theory("var r(S,S)\nA[i,j:S2] r(i,j)\n", k)
    th_g = oracle.Theory("var r(S,S)\nA[i,j:S | i!=j] r(i,j)\n", k)
    th_e = oracle.Theory("var r(S,S)\nE[i:S].A[j:S] r(i,j)\n", k)
    rng = np.random.default_rng(0)
    for j in rng.integers(0, 1 << 16, 300):
        j = int(j)
        rel = [[(j >> (i * k + l)) & 1 for l in range(k)] for i in range(k)]
        off = int(all(rel[i][l] for i in range(k) for l in range(k) if i != l))
        assert th_s2.eval(j) == off and th_g.eval(j) == off
        assert th_e.eval(j) == int(any(all(rel[i]) for i in range(k)))


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_relation_families_vs_brute_force(k):
    assert oracle.Theory(W.posets(k).text, k).count() == C.count_relations(k, "poset")
    assert oracle.Theory(W.equivalences(k).text, k).count() == C.count_relations(k, "equiv")
    assert oracle.Theory(W.transitive(k).text, k).count() == C.count_relations(k, "transitive")
    assert oracle.Theory(W.graphs(k).text, k).count() == C.count_relations(k, "graph")


def test_closed_forms():
    assert [oracle.Theory(W.posets(k).text, k).count() for k in (3, 4)] == [19, 219]
    assert oracle.Theory(W.posets(5).text, 5).count_par(0, 1 << 25) == 4231
    assert [oracle.Theory(W.equivalences(k).text, k).count() for k in range(1, 5)] == \
        [C.bell(k) for k in range(1, 5)] == [1, 2, 5, 15]
    assert oracle.Theory(W.equivalences(5).text, 5).count_par(0, 1 << 25) == C.bell(5) == 52
    assert [oracle.Theory(W.graphs(k).text, k).count() for k in (2, 3, 4)] == \
        [C.labelled_graphs(k) for k in (2, 3, 4)]
    assert C.count_posets_backtrack(4) == 219


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_triangle_free_vs_brute_force(k):
    assert oracle.Theory(W.triangle_free(k).text, k).count() == C.count_triangle_free(k)


@pytest.mark.parametrize("k,seed", [(3, 11), (4, 3), (4, 12), (5, 7)])
def test_automorphisms_vs_permutations(k, seed):
    wl = W.automorphisms(k, seed)
    th = oracle.Theory(wl.text, k)
    got = th.count_par(0, 1 << wl.n) if wl.n > 16 else th.count()
    assert got == C.count_automorphisms(W.random_graph_bits(k, seed), k)


def test_models_decode_to_structures():
    # each model of the poset theory, decoded by h (Sec. 3.2), is a partial order
    th = oracle.Theory(W.posets(3).text, 3)
    models, total = th.models(100)
    assert total == 19 and len(models) == 19
    for j in models:
        j = int(j)
        r = [[(j >> (i * 3 + l)) & 1 for l in range(3)] for i in range(3)]
        assert all(r[i][i] for i in range(3))
        assert all(not (r[i][l] and r[l][i]) for i in range(3) for l in range(3) if i != l)
        assert all((not (r[a][b] and r[b][c])) or r[a][c]
                   for a, b, c in itertools.product(range(3), repeat=3))


@pytest.mark.parametrize("n,seed", [(8, 1), (12, 2), (14, 3)])
def test_complement_and_shannon(n, seed):
    wl = W.cnf3(n, seed)
    th = oracle.Theory(wl.text, wl.k)
    body = [ln for ln in wl.text.splitlines()[1:] if ln.strip()]
    neg = oracle.Theory("var x(S)\n~(" + " & ".join(f"({c})" for c in body) + ")\n", wl.k)
    cnt = th.count()
    assert cnt + neg.count() == 1 << n
    for v in (0, n // 2, n - 1):
        assert th.count_cube(1 << v, 0) + th.count_cube(1 << v, 1 << v) == cnt
    # a cube count equals the brute-force count of the assignments in it
    mask, vals = 0b1011, 0b0010
    assert th.count_cube(mask, vals) == sum(th.eval(j) for j in range(1 << n) if (j & mask) == vals)


def test_range_count_and_table_agree():
    wl = W.cnf3(11, 9)
    th = oracle.Theory(wl.text, wl.k)
    t = th.table()
    assert sum(bin(int(w)).count("1") for w in t) == th.count()
    assert th.count(0, 1000) + th.count(1000, 2048) == th.count()
    models, total = th.models(5, 100, 2000)
    assert total == th.count(100, 2000)
    assert list(models) == [j for j in range(100, 2000) if th.eval(j)][:5]


@pytest.mark.parametrize("text,k", [
    ("var r(S,S)\nA[i:S] r(i,j)\n", 3),          # unbound index
    ("var e(S<S)\nA[a,b:S2] e(a,b)\n", 3),       # names e(b,a), b>a
    ("var r(S,S)\nr(1)\n", 3),                   # wrong arity
    ("var x\nx &\n", 1),                         # syntax
    ("var x\ny\n", 1),                           # undeclared
    ("const E(S,S) = 0101\nE(0,0)\n", 3),        # wrong bit count
])
def test_rejects_bad_text(text, k):
    with pytest.raises(oracle.OracleError):
        oracle.Theory(text, k)


def test_known_small_counts():
    # labelled transitive relations on 2..4 points and triangle-free graphs on
    # 3..5 vertices (both also fixed by the brute-force tests above)
    assert [oracle.Theory(W.transitive(k).text, k).count() for k in (2, 3, 4)] == [13, 171, 3994]
    assert [oracle.Theory(W.triangle_free(k).text, k).count() for k in (3, 4, 5)] == [7, 41, 388]


def test_backtracking_counters_match_brute_force_and_oracle():
    # the C backtracking counters used as full-size pins (n = 36) agree with
    # brute force and with the oracle wherever those finish
    for k in range(1, 5):
        assert C.count_transitive_backtrack(k) == C.count_relations(k, "transitive")
    for k in range(3, 8):
        assert C.count_triangle_free_backtrack(k) == C.count_triangle_free(k)
    assert C.count_transitive_backtrack(5) == oracle.Theory(W.transitive(5).text, 5).count_par(0, 1 << 25)
    assert C.count_triangle_free_backtrack(7) == oracle.Theory(W.triangle_free(7).text, 7).count()


def test_c_poset_counter_matches_brute_force_and_oracle():
    for k in range(1, 5):
        assert C.count_posets_c(k) == C.count_relations(k, "poset")
    assert C.count_posets_c(5) == 4231
