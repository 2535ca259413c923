"""GPU: the persistent batched launch (fbg_batch_*) against single counts and
the oracle.  Counts are exact integers: bit-exact equality."""
import numpy as np
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def small_mix(count, seed):
    """The batch families at sizes the oracle finishes quickly."""
    rng = W.SplitMix64(seed)
    out = []
    for _ in range(count):
        f = rng.below(5)
        if f == 0:
            out.append(W.equivalences(1 + rng.below(4)))
        elif f == 1:
            out.append(W.posets(1 + rng.below(4)))
        elif f == 2:
            out.append(W.triangle_free(3 + rng.below(4)))
        elif f == 3:
            out.append(W.cnf3(4 + rng.below(15), seed=rng.next()))
        else:
            out.append(W.transitive(2 + rng.below(3)))
    return out


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("max_item_units", [0, 1, 3])
def test_batch_equals_oracle(use_graph, max_item_units):
    mix = small_mix(300, 17)
    want = [oracle.Theory(w.text, w.k).count() for w in mix]
    progs = [F.compile(w.text, w.k) for w in mix]
    b = F.Batch(progs, max_item_units=max_item_units, use_graph=use_graph)
    for _ in range(3):                      # graph replays give the same counts
        b.run()
        got = b.results()
        assert [int(x) for x in got] == want


def test_batch_mix_matches_single_counts():
    """A slice of the 4096-formula mix (including n = 36 formulas): the batch
    equals one fbg_count per formula."""
    mix = W.batch_mix(4096, 2)
    sel = mix[:160] + [w for w in mix if w.n == 36][:4]
    progs = [F.compile(w.text, w.k) for w in sel]
    single = [F.compile(w.text, w.k).set_option(L.OPT_ENGINE, L.ENGINE_INTERP).count() for w in sel]
    b = F.Batch(progs)
    b.run()
    assert [int(x) for x in b.results()] == single
    items, units, grid = b.info()
    assert items >= len(sel) and units >= len(sel) and grid > 0


def test_batch_single_program_and_errors():
    p = F.compile(W.posets(4).text, 4)
    b = F.Batch([p])
    b.run()
    assert int(b.results()[0]) == 219
    with pytest.raises(L.FbgError):
        F.Batch([])
