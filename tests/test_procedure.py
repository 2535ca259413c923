"""The counting procedure of Sec. 3.4 (CPU): c-partition counts against the
closed forms of Sec. 3.4 and Sec. 5.2, and the procedure's l_{T,n} for
bounded posets against direct counts and the killed family of Sec. 5.2."""
import math

import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import procedure as P
from paper_1310_6978_b300 import workloads as W

import kernel_model as KM
from oracle import counters as C


def oracle_counter(wls):
    out = []
    for w in wls:
        th = oracle.Theory(w.text, w.k)
        out.append(th.count() if th.n <= 22 else th.count_par(0, 1 << th.n))
    return out


def model_counter(wls):
    return [KM.lut_program_count(F.compile(w.text, w.k).debug_dump(0)) for w in wls]


@pytest.mark.parametrize("n,m", [(1, 1), (3, 2), (4, 3), (5, 5), (6, 2), (7, 4)])
def test_c_partitions_match_closed_form(n, m):
    parts = list(P.c_partitions(n, m))
    assert len(parts) == len(set(parts)) == P.c_partition_count(n, m)
    assert all(sum(a) == n and len(a) == m for a in parts)


@pytest.mark.parametrize("n", range(3, 10))
def test_layer_partitions_are_2_to_the_n_minus_3(n):
    assert len(list(P.compositions(n - 2))) == 2 ** (n - 3)


def test_multinomial_weights_sum_to_ordered_set_partitions():
    # sum over compositions of the weights = ordered set partitions (Fubini numbers)
    fubini = [1, 1, 3, 13, 75, 541, 4683]
    for n in range(1, 7):
        assert sum(P.multinomial_weight(a) for a in P.compositions(n)) == fubini[n]


@pytest.mark.parametrize("n", [3, 4, 5])
def test_procedure_equals_direct_count(n):
    direct = oracle.Theory(W.bounded_posets(n).text, n)
    l_direct = direct.count() if n * n <= 20 else direct.count_par(0, 1 << (n * n))
    l_proc, detail = P.count_bounded_posets_by_layers(n, oracle_counter)
    assert l_proc == l_direct
    assert len(detail) == 2 ** (n - 3)


@pytest.mark.parametrize("n", [5, 6])
def test_procedure_on_compiled_programs_equals_killed_family(n):
    # the compiled programs (CPU model of the specialised kernel) give the same
    # l_{T,n} as n(n-1) |K| with K the killed family of Sec. 5.2
    l_proc, _ = P.count_bounded_posets_by_layers(n, model_counter)
    K = oracle_counter([W.bounded_posets_killed(n)])[0]
    assert l_proc == n * (n - 1) * K


def test_special_element_posets_pinned():
    # the SO.txt theory of Sec. 4.2: brute force over relations (k <= 4), the
    # backtracking counter, and the oracle agree
    for k in range(1, 5):
        w = W.posets_special(k)
        th = oracle.Theory(w.text, k)
        assert th.n == k * k - k
        assert th.count() == C.count_posets_special_brute(k) == C.count_posets_special_c(k)
    assert [C.count_posets_special_c(k) for k in (3, 4)] == [12, 116]


def test_partition_kills_follow_S():
    comps = P.canonical_components((2, 1))
    assert comps == [[0, 1], [2]]
    kills = P.partition_kills(comps, P.MINIMAL_S, "p")
    # S_11 = ~R(x,y) on the two minimal elements; S_12 = ~R(y,x): p(2,0), p(2,1) = 0
    assert sorted(kills) == sorted(["~p(0,1)", "~p(1,0)", "~p(2,0)", "~p(2,1)"])
    with pytest.raises(ValueError):
        P.partition_kills([[0, 1]], {(1, 1): "R(x,z)"}, "p")


@pytest.mark.parametrize("k", [2, 3, 4])
def test_general_procedure_on_two_theories_equals_direct_counts(k):
    """The counting procedure of Sec. 3.4 with the minimal / non-minimal
    partition reproduces the direct counts of partial orders (reflexivity
    killed) and of partial orders with a special element (SO.txt)."""
    for w, rel in ((W.posets_special(k), "p"), (W.posets_reflexivity_killed(k), "r")):
        direct = oracle_counter([w])[0]
        l, detail = P.count_by_partition(w.text, k, 2, lambda c, x: P.minimal_theta(c, x, rel), P.MINIMAL_S,
                                         oracle_counter, rel=rel)
        assert l == direct
        assert len(detail) == P.c_partition_count(k, 2)
        # no model has zero minimal elements
        assert [c for a, _, c in detail if a[0] == 0] == [0]
