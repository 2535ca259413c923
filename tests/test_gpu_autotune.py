"""GPU: the autotuner picks a kernel shape; results stay exact."""
import numpy as np
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import tuning
from paper_1310_6978_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_autotune_count_keeps_exact_counts():
    wl = W.cnf3(26, 3)
    th = oracle.Theory(wl.text, wl.k)
    p = F.compile(wl.text, wl.k)
    shape = p.autotune(0, reps=1)
    assert shape["trials"] >= 5 and shape["best_ms"] > 0
    assert p.count() == th.count_par(0, 1 << 26)
    q = F.compile(wl.text, wl.k).apply_shape(shape)
    assert q.count() == p.count()


def test_autotune_table_keeps_exact_table():
    wl = W.triangle_free(7)
    th = oracle.Theory(wl.text, wl.k)
    p = F.compile(wl.text, wl.k)
    shape = p.autotune(1, reps=1)
    t = torch.zeros(p.table_words(), dtype=torch.int64, device="cuda")
    p.truth_table(t)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy().view(np.uint64), th.table())
    cache = {}
    r = F.compile(wl.text, wl.k)
    assert tuning.ensure(r, 1, cache, tune=False) is None
    cache[tuning.key(wl.text, wl.k, 1)] = shape
    assert tuning.ensure(r, 1, cache) == shape
