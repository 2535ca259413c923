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
