"""GPU: programs compiled again from the same text share the host compiler's
products (the grounded theory, the kernel build: fbg_debug_host_caches) and
count exactly as the first one did; a different shape option is a different
build."""
import pytest

import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W
from oracle import counters as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_recompiled_text_reuses_builds_and_counts_the_same():
    F.host_caches(clear=True)
    wl = W.transitive(5)
    want = C.count_transitive_backtrack(5)
    a = F.compile(wl.text, wl.k)
    assert a.count() == want
    s0 = F.host_caches()
    b = F.compile(wl.text, wl.k)
    assert b.count() == want
    s1 = F.host_caches()
    assert s1["compile"]["hits"] == s0["compile"]["hits"] + 1
    assert s1["jit_build"]["hits"] == s0["jit_build"]["hits"] + 1
    assert s1["jit_build"]["misses"] == s0["jit_build"]["misses"]
    # another shape: a new build, the same count
    c = F.compile(wl.text, wl.k).set_option(L.OPT_REGS_LOG2, 1)
    assert c.count() == want
    assert F.host_caches()["jit_build"]["misses"] == s1["jit_build"]["misses"] + 1
    # the interpreter build is shared too
    d = F.compile(wl.text, wl.k).set_option(L.OPT_ENGINE, L.ENGINE_INTERP)
    e = F.compile(wl.text, wl.k).set_option(L.OPT_ENGINE, L.ENGINE_INTERP)
    assert d.count() == e.count() == want
    assert F.host_caches()["interp_build"]["hits"] >= 1
    # freeing programs leaves the shared entries usable
    del a, b, c, d, e
    assert F.compile(wl.text, wl.k).count() == want
