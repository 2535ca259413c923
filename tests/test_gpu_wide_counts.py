"""GPU: counts that reach the top of the unsigned 64-bit range.

A tautology over n letters has 2^n models (every position of its truth
vector is 1, Prop. 2.2), so at n = 63 the count is 2^63: it must come back
through fbg_count, fbg_count_async, fbg_count_range and fbg_count_units as an
unsigned value on both engines.  The Reduction (Sec. 4.1) folds such a
formula to a constant, so these counts need no evaluation of 2^63 points.
"""
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


TAUT = "var x(S)\nx(0) | ~x(0)\n"
CONTRA = "var x(S)\nx(0) & ~x(0)\n"


@pytest.mark.parametrize("engine", [L.ENGINE_JIT, L.ENGINE_INTERP])
@pytest.mark.parametrize("n", [62, 63])
def test_tautology_counts_are_unsigned(engine, n):
    p = F.compile(TAUT, n).set_option(L.OPT_ENGINE, engine)
    assert p.n == n
    assert p.count() == 1 << n
    out = torch.full((3,), -7, dtype=torch.int64, device="cuda")
    p.count_async(out[1:2])
    torch.cuda.synchronize()
    assert F.read_counts(out) == [(1 << 64) - 7, 1 << n, (1 << 64) - 7]
    _, nunits = p.unit_vars()
    half = nunits // 2
    assert p.count_range(0, half) + p.count_range(half, nunits) == 1 << n
    assert p.count_range(3, 3) == 0


def test_tautology_per_unit_counts():
    p = F.compile(TAUT, 40)
    _, nunits = p.unit_vars()
    uc = torch.zeros(nunits, dtype=torch.int64, device="cuda")
    p.count_units(uc)
    torch.cuda.synchronize()
    assert set(F.read_counts(uc)) == {(1 << 40) // nunits}


def test_contradiction_and_killed_tautology():
    assert F.compile(CONTRA, 63).count() == 0
    # killing x(0) leaves 62 free letters and the constant 1 (Sec. 3.3)
    text = "var x(S)\nassume x(0)\nx(0)\n"
    p = F.compile(text, 63)
    assert p.n == 62
    assert p.count() == 1 << 62
    # the oracle agrees on a small instance of the same texts
    for k in (3, 5):
        assert F.compile(text, k).count() == oracle.Theory(text, k).count() == 1 << (k - 1)
        assert F.compile(TAUT, k).count() == oracle.Theory(TAUT, k).count() == 1 << k
