"""The generated CUDA source of the specialised kernels, compiled as host C++
(tests/jit_host.py) and checked against the oracle: counts and truth tables
bit-exact, under several layouts.  No GPU needed."""
import numpy as np
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

import jit_host

CASES = [W.BAEQU4, W.POSET3, W.posets(4), W.transitive(4), W.equivalences(4), W.triangle_free(6),
         W.automorphisms(4, 3), W.cnf3(14, 2), W.cnf3(18, 5), W.single_var(6, 5), W.minterm(3, 6),
         W.Workload("xor", 0, "var a, b, c, d, e, f, g, h\n(a ^ b ^ c) | (d & ~e) <-> (f -> g ^ h)\n", 1, 8),
         W.Workload("unsat", 0, "var a, b, c, d, e, f, g\n(a & ~a) | (b & 0)\n", 1, 7),
         # function symbols (Sec. 3.1)
         W.semigroups(2), W.latin_squares(3, first_row=True), W.reduced_latin_squares(4), W.groups(2),
         W.Workload("image", 3, "var r(S)\nfun f(S)\nA[x:S] r(f(x))\n", 3, 12),
         W.Workload("inj", 3, "fun f(S)\nA[x,y:S] (x != y -> f(x) != f(y))\n", 3, 9),
         W.Workload("nested", 2, "var r(S,S)\nfun f(S), c\nA[x:S] (r(x, f(f(x))) | f(c) = x)\n", 2, 10)]

LAYOUTS = [
    {},
    {L.OPT_REGS_LOG2: 1, L.OPT_WARPS_LOG2: 0, L.OPT_UNIT_BITS: 1, L.OPT_LOOP_LEVEL_BITS: 1},
    {L.OPT_REGS_LOG2: 3, L.OPT_WARPS_LOG2: 1, L.OPT_UNIT_BITS: 2, L.OPT_LOOP_LEVEL_BITS: 2},
    {L.OPT_PRUNE: 0, L.OPT_WARPS_LOG2: 0, L.OPT_UNIT_BITS: 1, L.OPT_LOOP_LEVEL_BITS: 2},
    {L.OPT_REGS_LOG2: 2, L.OPT_WARPS_LOG2: 1, L.OPT_UNIT_BITS: 2, L.OPT_LOOP_LEVEL_BITS: 1, L.OPT_INNER_BITS: 3},
]


@pytest.mark.parametrize("wl", CASES, ids=lambda w: f"{w.family}{w.param}n{w.n}")
@pytest.mark.parametrize("li", range(len(LAYOUTS)))
def test_generated_source_matches_oracle(wl, li):
    th = oracle.Theory(wl.text, wl.k)
    p = F.compile(wl.text, wl.k)
    for k, v in LAYOUTS[li].items():
        p.set_option(k, v)
    for mode in (0, 1):
        d0 = p.debug_dump(mode)
        d = d0["layout"]
        block = 32 if d["lane_bits"] < 5 else 32 << d["warp_bits"]
        nunits = 1 << d["unit_bits"]
        src = p.source(mode)
        if mode == 0:
            assert jit_host.run_count(src, block, nunits) == th.count()
            # a scheduled launch: every (unit, warp slice) item once, in a shuffled order
            items = nunits << d["warp_bits"]
            perm = np.random.default_rng(items).permutation(items).astype(np.uint32)
            assert jit_host.run_count(src, block, nunits, perm) == th.count()
            assert jit_host.run_count(src, block, nunits, perm, self_reset=True) == th.count()
            # only the items whose unit and warp conjuncts hold (the list full-range counts use)
            if "alive_items" in d0:
                live = np.array(d0["alive_items"], dtype=np.uint32)
                assert jit_host.run_count(src, block, nunits, live, self_reset=True) == th.count()
            # items handed out as pieces over the first loop level (entry
            # item | s << 28 | q << 24): every item in 2^s pieces, and a mix
            sb = d["split_bits"]
            if sb:
                for s in sorted({1, sb}):
                    whole = np.repeat(np.arange(items, dtype=np.uint32), 1 << s)
                    q = np.tile(np.arange(1 << s, dtype=np.uint32), items)
                    split = whole | np.uint32(s << 28) | (q << np.uint32(24))
                    split = split[np.random.default_rng(s).permutation(len(split))]
                    assert jit_host.run_count(src, block, nunits, split, self_reset=True) == th.count()
                ent = []
                for t in range(items):
                    if t % 3:
                        ent.append(t)
                    else:
                        ent += [t | (sb << 28) | (q << 24) for q in range(1 << sb)]
                assert jit_host.run_count(src, block, nunits, np.array(ent[::-1], dtype=np.uint32)) == th.count()
            else:
                assert len(d["loop_bits"]) <= 1
        else:
            assert np.array_equal(jit_host.run_table(src, block, nunits, p.table_words()), th.table())
