"""Host compile cache (no GPU): the same (text, domain size) compiles once;
programs from it are independent handles with the same letters."""
import pytest

import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W


def test_compile_cache_hits_and_keys():
    F.host_caches(clear=True)
    a = F.compile(W.POSET3.text, 3)
    b = F.compile(W.POSET3.text, 3)
    c = F.compile(W.POSET3.text, 4)          # another domain size: another theory
    st = F.host_caches()["compile"]
    assert st["hits"] >= 1 and st["misses"] >= 2
    assert a.n == b.n == 9 and c.n == 16
    assert [a.var_name(i) for i in range(9)] == [b.var_name(i) for i in range(9)]
    del a
    assert b.var_name(8) == "r(2,2)"
    with pytest.raises(L.FbgError):
        F.compile("var x\nx &\n", 1)
    with pytest.raises(L.FbgError):
        F.compile("var x\nx &\n", 1)          # errors are not cached as programs


def test_build_can_leave_no_live_unit():
    """Random 3-CNF n = 30 at ratio 8 (seed 1): at the server's count layout
    (2^20 units requested) the conjuncts over unit letters kill every unit at
    build time, which the server finishes without a launch; at ratio 6 some
    units survive."""
    from paper_1310_6978_b300 import _lib as L
    from paper_1310_6978_b300 import workloads as W
    for ratio, dead in ((8.0, True), (6.0, False)):
        wl = W.cnf3(30, 1, ratio)
        p = F.compile(wl.text, wl.k).set_option(L.OPT_ENGINE, L.ENGINE_INTERP).set_option(L.OPT_UNIT_BITS, 20)
        d = p.debug_dump(2)
        assert p.stats().luts > 0
        assert (d["live_units"] == 0) == dead and d["live_units"] >= 0
