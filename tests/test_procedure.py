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
