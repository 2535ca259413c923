"""The layout of the specialised model-list kernel (no GPU).

Its work items (unit u, warp slice w) must each cover one interval of
assignment integers, in the order of the item index u << wb | w, and the
loop nest inside an item must run through the interval in ascending order
(outer loop levels on higher bits, the unrolled innermost level above the
lanes), so that the per-item counts, their prefix sums and the in-order writes
give the models of Sec. 4.2 in ascending j.
"""
import pytest

import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

SHAPES = [{}, {L.OPT_REGS_LOG2: 1, L.OPT_WARPS_LOG2: 0, L.OPT_UNIT_BITS: 1, L.OPT_LOOP_LEVEL_BITS: 1},
          {L.OPT_REGS_LOG2: 3, L.OPT_WARPS_LOG2: 2, L.OPT_UNIT_BITS: 2, L.OPT_LOOP_LEVEL_BITS: 2},
          {L.OPT_INNER_BITS: 3, L.OPT_UNIT_BITS: 5}]


@pytest.mark.parametrize("wl", [W.POSET3, W.posets(4), W.cnf3(20, 4), W.TRANSITIVE6, W.cnf3(38, 5), W.single_var(7, 6)],
                         ids=lambda w: f"{w.family}{w.param}n{w.n}")
@pytest.mark.parametrize("si", range(len(SHAPES)))
def test_items_are_ascending_intervals(wl, si):
    p = F.compile(wl.text, wl.k)
    for k, v in SHAPES[si].items():
        p.set_option(k, v)
    lay = p.debug_dump(4)["layout"]
    n = lay["n"]
    pos_of_var = lay["pos_of_var"]
    var_of_pos = [0] * n
    for v, pos in enumerate(pos_of_var):
        var_of_pos[pos] = v
    assert sorted(pos_of_var) == list(range(n))
    ub, wb, lb, r = lay["unit_bits"], lay["warp_bits"], lay["lane_bits"], lay["r"]
    top = n - ub
    # units and the warp slice are the top letters, in place
    for b in range(ub):
        assert var_of_pos[top + b] == top + b
    w0 = 5 + r + lb if n > 5 else 0
    for b in range(wb):
        assert var_of_pos[w0 + b] == top - wb + b
    # lanes, registers and in-word bits keep their own letters
    for pos in range(min(n, w0)):
        assert var_of_pos[pos] == pos
    # loop levels: each level's bits map to consecutive letters, the outer
    # levels to higher letters, all just below the warp slice
    expect = top - wb
    for bits, lp in zip(lay["loop_bits"], lay["loop_pos"]):
        expect -= bits
        assert [var_of_pos[lp + b] for b in range(bits)] == list(range(expect, expect + bits))
    assert expect == w0
    # the source of that layout is the one the kernel build compiles
    src = p.source(2)
    assert "fbg_jit_enum" in src and "fbg_unit_enum" in src
