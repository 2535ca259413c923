"""Random formulas through the whole host compiler (no GPU).

Seeded random propositional formulas over 6 to 13 letters -- nested
~ & | ^ -> <-> with shared subterms and constants -- are compiled, and the
generated CUDA source of the specialised count and table kernels (compiled
as host C++, tests/jit_host.py) and the interpreter bytecode (CPU model,
tests/kernel_model.py) must give the oracle's counts and tables bit for bit,
under several layouts.  This exercises the Reduction, the LOP3 mapping, the
folding and the merge of folded LUT chains, the block slots of the
interpreter and the pruning on formulas nobody wrote by hand.
"""
import numpy as np
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

import jit_host
import kernel_model as KM

LAYOUTS = [
    {},
    {L.OPT_REGS_LOG2: 1, L.OPT_WARPS_LOG2: 0, L.OPT_UNIT_BITS: 1, L.OPT_LOOP_LEVEL_BITS: 1},
    {L.OPT_REGS_LOG2: 3, L.OPT_WARPS_LOG2: 1, L.OPT_UNIT_BITS: 2, L.OPT_LOOP_LEVEL_BITS: 2, L.OPT_INNER_BITS: 2},
    {L.OPT_REGS_LOG2: 2, L.OPT_WARPS_LOG2: 0, L.OPT_UNIT_BITS: 2, L.OPT_LOOP_LEVEL_BITS: 1, L.OPT_POPC_COST: 0},
]


def random_formula(seed: int):
    """Formula text over n letters v0..v{n-1}: a conjunction of a few random
    clauses and one random expression tree that reuses subterms."""
    rng = W.SplitMix64(seed)
    n = 6 + rng.below(8)
    names = [f"v{i}" for i in range(n)]
    pool = list(names)

    def expr(depth):
        if depth == 0 or rng.below(4) == 0:
            leaf = pool[rng.below(len(pool))] if rng.below(8) else ("1" if rng.below(2) else "0")
            return ("~" + leaf) if rng.below(3) == 0 and leaf not in ("0", "1") else leaf
        op = ["&", "|", "^", "->", "<->"][rng.below(5)]
        e = f"({expr(depth - 1)} {op} {expr(depth - 1)})"
        if rng.below(3) == 0:
            pool.append(e)               # reuse it below: a shared subterm
        return e

    lines = ["var " + ", ".join(names)]
    for _ in range(rng.below(5)):
        lits = [("~" if rng.below(2) else "") + names[rng.below(n)] for _ in range(2 + rng.below(2))]
        lines.append(" | ".join(lits))
    lines.append(expr(4))
    return "\n".join(lines) + "\n", n


@pytest.mark.parametrize("seed", range(80))
def test_random_formula_compiles_to_the_oracle(seed):
    text, n = random_formula(seed * 7919 + 1)
    th = oracle.Theory(text, 1)
    assert th.n == n
    want_count, want_table = th.count(), th.table()
    li = seed % len(LAYOUTS)
    p = F.compile(text, 1)
    for k, v in LAYOUTS[li].items():
        p.set_option(k, v)
    for mode in (0, 1):
        d = p.debug_dump(mode)["layout"]
        block = 32 if d["lane_bits"] < 5 else 32 << d["warp_bits"]
        nunits = 1 << d["unit_bits"]
        src = p.source(mode)
        if mode == 0:
            assert jit_host.run_count(src, block, nunits) == want_count
        else:
            assert np.array_equal(jit_host.run_table(src, block, nunits, p.table_words()), want_table)
    assert KM.interp_count(p.debug_dump(2)) == want_count
    assert np.array_equal(KM.interp_table(p.debug_dump(3)), want_table)
