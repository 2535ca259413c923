"""The measured lop3.b32 rate lands near the nominal integer-logic peak the
roofline uses (148 SMs x 64 lanes/clk x the SM clock)."""
import pytest
import torch

import paper_1310_6978_b300 as F

pytestmark = pytest.mark.gpu


def test_lop3_rate_near_nominal_peak():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 64 * 2.032e9 / 1e12
    rate = F.probe_lop3_rate()
    # below the top clock the rate drops in proportion; far above it the probe would be wrong
    assert 0.5 * nominal < rate < 1.1 * nominal, (rate, nominal)


@pytest.mark.parametrize("prune", [0, 1])
@pytest.mark.parametrize("case", ["posets5_u2", "trifree9"])
def test_exec_stats_follow_the_layout(case, prune):
    """The executed-work counters behind the bench's roofline: executed lane
    operations are the level iterations times the lane-varying lop3 per level
    (x 32 lanes); without pruning every level runs its closed-form number of
    times and executed + 32 x uniform, less level 0 (whose count depends on
    the work chunks), is the nominal work."""
    from paper_1310_6978_b300 import _lib as L
    from paper_1310_6978_b300 import workloads as W
    wl, opts, want = {"posets5_u2": (W.posets(5), {L.OPT_UNIT_BITS: 2}, 4231),
                      "trifree9": (W.TRIFREE9, {}, 246348115)}[case]
    p = F.compile(wl.text, wl.k)
    for k, v in opts.items():
        p.set_option(k, v)
    p.set_option(L.OPT_PRUNE, prune)
    p.set_option(L.OPT_STATS, 1)
    assert p.count() == want
    es = p.exec_stats()
    st = p.stats()
    nl = st.nlevels
    ops = list(st.lop3_per_level)[:nl]
    loops = list(st.loop_bits)[:nl - 2]
    it = list(es.level_iters)[:nl]
    assert es.lop3_executed == 32 * sum(i * o for i, o in zip(it, ops))
    # closed form: level 1 runs once per (unit, warp slice); a loop level
    # multiplies by its width; the innermost level, when it is emitted
    # unrolled (at most 5 bits), runs once per iteration of the level above
    closed = [None, (1 << st.unit_bits) << st.warp_bits]
    for lv in range(2, nl):
        unrolled = lv == nl - 1 and loops[-1] <= 5
        closed.append(closed[-1] if unrolled else closed[-1] << loops[lv - 2])
    for lv in range(1, nl):
        assert it[lv] <= closed[lv]
        if not prune:
            assert it[lv] == closed[lv], (lv, it, closed)
    if not prune:
        lhs = es.lop3_executed - 32 * it[0] * ops[0] + 32 * es.lop3_uniform
        assert abs(lhs - es.lop3_nominal) <= 1e-9 * es.lop3_nominal
    else:
        assert es.lop3_executed < es.lop3_nominal


def test_host_times_split_builds_from_counts():
    """fbg_debug_host_times: the first count builds the kernel (build time
    grows), a second count of the same program does not rebuild (build time
    unchanged, count time grows)."""
    from paper_1310_6978_b300 import workloads as W
    p = F.compile(W.posets(5).text, 5)
    assert p.debug_host_times() == (0.0, 0.0)
    assert p.count() == 4231
    b1, c1 = p.debug_host_times()
    assert b1 > 0 and c1 > 0
    assert p.count() == 4231
    b2, c2 = p.debug_host_times()
    assert b2 == b1 and c2 > c1


@pytest.mark.parametrize("prune", [0, 1])
def test_interpreter_exec_stats_follow_the_layout(prune):
    """The interpreter's level counters (units of 32 tiles): level 1 runs once
    per unit for each of the block's two 32-tile halves, a loop level
    multiplies by its width; without pruning every level runs that often and
    the executed lane operations (64 lop3.b32 per LUT and 32 tiles) of levels
    1.. are the nominal work."""
    from paper_1310_6978_b300 import _lib as L
    from paper_1310_6978_b300 import workloads as W
    wl = W.TRIFREE9
    p = F.compile(wl.text, wl.k).set_option(L.OPT_ENGINE, L.ENGINE_INTERP).set_option(L.OPT_UNIT_BITS, 14)
    p.set_option(L.OPT_PRUNE, prune)
    p.set_option(L.OPT_STATS, 1)
    assert p.count() == 246348115
    es = p.exec_stats()
    d = p.debug_dump(2)
    lev = d["levels"]
    nl = len(lev)
    it = list(es.level_iters)[:nl]
    luts = [l[1] - l[0] for l in lev]
    assert es.lop3_executed == 64 * sum(i * n for i, n in zip(it, luts))
    closed = [None, (1 << d["unit_bits"]) * 2]
    for lv in range(2, nl):
        closed.append(closed[-1] << lev[lv][2])
    for lv in range(1, nl):
        assert it[lv] <= closed[lv]
        if not prune:
            assert it[lv] == closed[lv], (lv, it, closed)
    if not prune:
        assert es.lop3_executed - 64 * it[0] * luts[0] == es.lop3_nominal
    else:
        assert es.lop3_executed < es.lop3_nominal
