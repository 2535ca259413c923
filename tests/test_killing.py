"""Killing variables (Sec. 3.3, the assumptions of Sec. 4.2) on the CPU: the
oracle and the compiled program (CPU models of both kernels) against closed
forms and the definable-constants identity l_{T,n} = n(n-1)|K| of Sec. 3.3
for the bounded posets of Sec. 5.2."""
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

import kernel_model as KM


def both_counts(wl):
    th = oracle.Theory(wl.text, wl.k)
    p = F.compile(wl.text, wl.k)
    assert p.n == th.n == wl.n
    c = th.count() if th.n <= 20 else th.count_par(0, 1 << th.n)
    assert KM.lut_program_count(p.debug_dump(0)) == c
    assert KM.interp_count(p.debug_dump(2)) == c
    return c


@pytest.mark.parametrize("k,want", [(2, 3), (3, 19), (4, 219)])
def test_reflexivity_killed_keeps_the_poset_count(k, want):
    # SO.txt: n^2 - n free letters once p(i,i) are killed
    assert both_counts(W.posets_reflexivity_killed(k)) == want


@pytest.mark.parametrize("k", [3, 4, 5])
def test_bounded_posets_definable_constants(k):
    # l_{T,n} = n(n-1) |K| (Sec. 3.3) with K the killed family of Sec. 5.2
    direct = oracle.Theory(W.bounded_posets(k).text, k)
    l_direct = direct.count() if k * k <= 20 else direct.count_par(0, 1 << (k * k))
    K = both_counts(W.bounded_posets_killed(k))
    assert l_direct == k * (k - 1) * K
    assert W.bounded_posets_killed(k).n == k * k - (5 * k - 6)


def test_small_bounded_poset_values():
    # n = 3: the middle element is forced (|K| = 1); n = 4: two middle
    # elements are ordered either way or incomparable (|K| = 3)
    assert both_counts(W.bounded_posets_killed(3)) == 1
    assert both_counts(W.bounded_posets_killed(4)) == 3


def test_later_assumptions_override_earlier_ones():
    text = "var r(S,S)\nassume A[i:S] r(i,i)\nassume ~r(0,0)\nr(0,1) | r(1,0) | r(0,0)\n"
    th = oracle.Theory(text, 2)
    p = F.compile(text, 2)
    assert th.n == p.n == 2
    assert [p.var_name(i) for i in range(2)] == ["r(0,1)", "r(1,0)"]
    assert th.count() == KM.lut_program_count(p.debug_dump(0)) == 3


@pytest.mark.parametrize("text", ["var x, y\nassume x | y\nx\n", "var x, y\nassume ~(x & y)\nx\n",
                                  "var x\nconst C(S) = 1\nassume C(0)\nx\n"])
def test_assume_must_be_literals(text):
    with pytest.raises(L.FbgError):
        F.compile(text, 1)
    with pytest.raises(oracle.OracleError):
        oracle.Theory(text, 1)
