"""Build-time pruning (alive_items): an item (unit u, warp slice w) marked
dead must have no models.  Checked against the oracle: the sub-cube with
the item's unit and warp letters fixed to the item's bits counts 0, and the
live items together hold every model."""
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

CASES = [W.posets(4), W.transitive(4), W.equivalences(4), W.triangle_free(6), W.automorphisms(4, 3),
         W.cnf3(18, 5), W.semigroups(2), W.latin_squares(3, first_row=True), W.bounded_posets_killed(6)]


@pytest.mark.parametrize("wl", CASES, ids=lambda w: f"{w.family}{w.param}")
@pytest.mark.parametrize("shape", [{L.OPT_UNIT_BITS: 3, L.OPT_WARPS_LOG2: 1}, {L.OPT_UNIT_BITS: 5, L.OPT_WARPS_LOG2: 2},
                                   {L.OPT_UNIT_BITS: 9, L.OPT_WARPS_LOG2: 2, L.OPT_REGS_LOG2: 1}])
def test_dead_items_have_no_models(wl, shape, par=False):
    p = F.compile(wl.text, wl.k)
    for k, v in shape.items():
        p.set_option(k, v)
    d = p.debug_dump(0)
    lay = d["layout"]
    if "alive_items" not in d:
        pytest.skip("no conjunct over unit and warp letters")
    th = oracle.Theory(wl.text, wl.k)
    pos_of_var = lay["pos_of_var"]
    var_of_pos = {pos: v for v, pos in enumerate(pos_of_var)}
    wb, ub = lay["warp_bits"], lay["unit_bits"]
    first_warp = 5 + lay["r"] + lay["lane_bits"]
    first_unit = lay["first_unit_pos"]
    item_vars = [var_of_pos[first_warp + b] for b in range(wb)] + [var_of_pos[first_unit + b] for b in range(ub)]
    mask = sum(1 << v for v in item_vars)
    live = set(d["alive_items"])
    total = 0
    for t in range(1 << (ub + wb)):
        vals = sum(((t >> b) & 1) << v for b, v in enumerate(item_vars))
        c = th.count_cube_par(mask, vals) if par else th.count_cube(mask, vals)
        if t not in live:
            assert c == 0, (t, c)
        total += c
    assert total == (th.count_par(0, 1 << wl.n) if par else th.count())


@pytest.mark.parametrize("wl", [W.cnf3(24, 5), W.posets(5), W.triangle_free(7)], ids=lambda w: f"{w.family}{w.param}")
def test_dead_items_have_no_models_many_items(wl):
    """The same on item spaces of 2^8 to 2^11 items, where the word-index
    letters of a conjunct are gathered from the word number (several words,
    per-conjunct tables)."""
    test_dead_items_have_no_models(wl, {L.OPT_UNIT_BITS: 9, L.OPT_WARPS_LOG2: 2, L.OPT_REGS_LOG2: 1}, par=True)
