"""The host compiler checked against the oracle on the CPU (no GPU).

The compiled program (fbg_debug_dump) is run through CPU models of the two
kernels (tests/kernel_model.py): counts, truth tables and model lists must
equal the oracle's bit for bit, and every level's partial conjunction must
cover the formula value (so pruning is sound).  Options force small tiles,
few units and one-bit loop levels so that every level of the layout is used
at small n.
"""
import itertools

import numpy as np
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

import kernel_model as KM

CASES = [
    W.BAEQU4, W.posets(2), W.POSET3, W.posets(4), W.equivalences(3), W.equivalences(4), W.transitive(3),
    W.transitive(4), W.graphs(3), W.triangle_free(4), W.triangle_free(5), W.triangle_free(6),
    W.automorphisms(3, 11), W.automorphisms(4, 3), W.cnf3(7, 5), W.cnf3(12, 1), W.cnf3(14, 2), W.cnf3(16, 3),
    W.minterm(3, 5), W.single_var(7, 6),
    W.Workload("xor", 0, "var a, b, c, d, e, f, g, h\n(a ^ b ^ c) | (d & ~e) <-> (f -> g ^ h)\n", 1, 8),
    W.Workload("taut", 0, "var a, b, c\na | ~a\n", 1, 3),
    W.Workload("unsat", 0, "var a, b, c, d, e, f, g\n(a & ~a) | (b & 0)\n", 1, 7),
    W.Workload("one", 0, "var a\na\n", 1, 1),
    W.Workload("nested", 0, "var p(S,S)\nE[i:S] (A[j:S] p(i,j) | A[j:S | j!=i] ~p(j,i))\n", 3, 9),
]

OPTION_SETS = [
    {},
    {L.OPT_REGS_LOG2: 1, L.OPT_WARPS_LOG2: 0, L.OPT_UNIT_BITS: 1, L.OPT_LOOP_LEVEL_BITS: 1},
    {L.OPT_REGS_LOG2: 3, L.OPT_WARPS_LOG2: 0, L.OPT_UNIT_BITS: 2, L.OPT_LOOP_LEVEL_BITS: 2},
    {L.OPT_REGS_LOG2: 2, L.OPT_WARPS_LOG2: 1, L.OPT_UNIT_BITS: 0, L.OPT_LOOP_LEVEL_BITS: 1, L.OPT_SEARCH_ORDER: 0},
    {L.OPT_PRUNE: 0, L.OPT_WARPS_LOG2: 0, L.OPT_UNIT_BITS: 1, L.OPT_LOOP_LEVEL_BITS: 1},
]


def truth(wl):
    th = oracle.Theory(wl.text, wl.k)
    return th


@pytest.mark.parametrize("wl", CASES, ids=lambda w: f"{w.family}{w.param}n{w.n}")
@pytest.mark.parametrize("oi", range(len(OPTION_SETS)))
def test_lut_program_matches_oracle(wl, oi):
    th = truth(wl)
    p = F.compile(wl.text, wl.k)
    for k, v in OPTION_SETS[oi].items():
        p.set_option(k, v)
    assert p.n == th.n
    d0 = p.debug_dump(0)
    assert KM.lut_program_count(d0) == th.count()
    assert KM.lut_program_prune_sound(d0)
    d1 = p.debug_dump(1)
    assert d1["layout"]["pos_of_var"] == list(range(p.n))
    assert np.array_equal(KM.lut_program_table(d1), th.table())
    assert KM.lut_program_prune_sound(d1)


@pytest.mark.parametrize("wl", CASES, ids=lambda w: f"{w.family}{w.param}n{w.n}")
@pytest.mark.parametrize("oi", [0, 1, 4])
def test_interpreter_model_matches_oracle(wl, oi):
    th = truth(wl)
    p = F.compile(wl.text, wl.k)
    for k, v in OPTION_SETS[oi].items():
        if k in (L.OPT_REGS_LOG2, L.OPT_WARPS_LOG2):
            continue   # the interpreter has a fixed tile and block
        p.set_option(k, v)
    d2 = p.debug_dump(2)
    assert KM.interp_count(d2) == th.count()
    d3 = p.debug_dump(3)
    assert np.array_equal(KM.interp_table(d3), th.table())
    cap = 7
    models, total = KM.interp_models(d3, cap)
    om, ot = th.models(cap)
    assert total == ot and models == [int(x) for x in om]


def test_search_order_is_a_permutation_and_count_invariant():
    wl = W.transitive(4)
    p = F.compile(wl.text, wl.k)
    d = p.debug_dump(0)
    assert sorted(d["layout"]["pos_of_var"]) == list(range(16))
    assert d["layout"]["pos_of_var"] != list(range(16))   # the heuristic moved letters
    assert KM.lut_program_count(d) == 3994


def test_var_names_and_numbering():
    p = F.compile("var r(S,S), e(S<S)\nr(0,1) | e(0,2)\n", 3)
    assert p.n == 9 + 3
    assert [p.var_name(i) for i in (0, 5, 9, 10, 11)] == ["r(0,0)", "r(1,2)", "e(0,1)", "e(0,2)", "e(1,2)"]


@pytest.mark.parametrize("text,k", [
    ("var r(S,S)\nA[i:S] r(i,j)\n", 3),
    ("var e(S<S)\nA[a,b:S2] e(a,b)\n", 3),
    ("var r(S,S)\nr(1)\n", 3),
    ("var x\nx &\n", 1),
    ("var x\ny\n", 1),
    ("const E(S,S) = 0101\nE(0,0)\n", 3),
])
def test_compile_rejects_bad_text(text, k):
    with pytest.raises(L.FbgError) as ei:
        F.compile(text, k)
    assert ei.value.status == L.FBG_EPARSE


def test_too_many_letters():
    with pytest.raises(L.FbgError) as ei:
        F.compile("var r(S,S)\nr(0,0)\n", 9)
    assert ei.value.status == L.FBG_ETOOBIG


def test_dag_sharing_and_constant_removal():
    # constants vanish in the DAG (Reduction, Sec. 4.1); repeated clauses are shared
    a = F.compile("var a, b\n(a | 0) & (b | 0) & 1\n").stats()
    b = F.compile("var a, b\na & b\na & b\n").stats()
    assert a.luts == b.luts


@pytest.mark.parametrize("seed", [0, 1, 2, 5])
def test_order_variants_keep_counts(seed):
    # the seeded tie-break variants of the count order (FBG_OPT_ORDER_SEED)
    # place the letters differently and leave every count unchanged
    import oracle
    from paper_1310_6978_b300 import _lib as L
    for wl in (W.triangle_free(6), W.posets(4), W.transitive(4), W.cnf3(14, 3)):
        p = F.compile(wl.text, wl.k).set_option(L.OPT_ORDER_SEED, seed)
        d = p.debug_dump(0)
        assert sorted(d["layout"]["pos_of_var"]) == list(range(wl.n))
        assert KM.lut_program_count(d) == oracle.Theory(wl.text, wl.k).count()
