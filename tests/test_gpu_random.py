"""GPU: the seeded random formulas of tests/test_random_formulas.py on the
real kernels -- counts, truth tables and model lists of the specialised
kernels and the interpreter against the oracle (exact)."""
import numpy as np
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L

from test_random_formulas import LAYOUTS, random_formula

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("seed", range(32))
def test_random_formula_on_the_gpu(seed):
    text, n = random_formula(seed * 7919 + 1)
    th = oracle.Theory(text, 1)
    want_models, want_total = th.models(1 << n)
    for engine in (L.ENGINE_JIT, L.ENGINE_INTERP):
        p = F.compile(text, 1).set_option(L.OPT_ENGINE, engine)
        if engine == L.ENGINE_JIT:
            for k, v in LAYOUTS[seed % len(LAYOUTS)].items():
                p.set_option(k, v)
        assert p.count() == want_total
        t = torch.full((p.table_words(),), -1, dtype=torch.int64, device="cuda")
        p.truth_table(t)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy().view(np.uint64), th.table())
        buf = torch.full((max(1, want_total),), -1, dtype=torch.int64, device="cuda")
        total, written = p.enumerate_models(buf, want_total)
        assert total == want_total == written
        assert np.array_equal(buf[:written].cpu().numpy().view(np.uint64), want_models)
