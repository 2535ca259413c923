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
@pytest.mark.parametrize("specialize", [False, True])
@pytest.mark.parametrize("max_item_units", [0, 1, 3])
def test_batch_equals_oracle(use_graph, specialize, max_item_units):
    mix = small_mix(300, 17)
    want = [oracle.Theory(w.text, w.k).count() for w in mix]
    progs = [F.compile(w.text, w.k) for w in mix]
    b = F.Batch(progs, max_item_units=max_item_units, use_graph=use_graph, specialize=specialize)
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
    info = b.info()
    assert info["items"] >= len(sel) and info["units"] >= len(sel) and info["grid"] > 0
    # the n = 36 equivalence formulas carry the work: specialised
    assert info["specialized"] >= 1
    kinds = b.program_kinds()
    assert all(kinds[i] == 1 for i, w in enumerate(sel) if w.n == 36)


def test_batch_mixes_specialised_and_interpreted():
    """Two heavy programs on specialised kernels (three instances each, on
    side streams), many light ones in the interpreter launch."""
    heavy = [W.transitive(5), W.equivalences(5)] * 3
    light = small_mix(80, 9)
    mix = heavy + light
    progs = [F.compile(w.text, w.k) for w in mix]
    b = F.Batch(progs, specialize=True)
    for _ in range(2):
        b.run()
        got = [int(x) for x in b.results()]
        assert got[:6] == [oracle.Theory(w.text, w.k).count_par(0, 1 << 25) for w in heavy]
        assert got[6:] == [oracle.Theory(w.text, w.k).count() for w in light]
    assert b.info()["specialized"] == 2
    assert b.program_kinds()[:6] == [1] * 6


def test_batch_single_program_and_errors():
    p = F.compile(W.posets(4).text, 4)
    b = F.Batch([p])
    b.run()
    assert int(b.results()[0]) == 219
    with pytest.raises(L.FbgError):
        F.Batch([])


def test_count_each_equals_oracle_on_both_engines():
    """fbg_count_each (one launch per program from C, the plain baseline of
    the batch) writes every program's count, on both engines."""
    mix = small_mix(40, 17)
    want = [oracle.Theory(w.text, w.k).count() for w in mix]
    for engine in (L.ENGINE_JIT, L.ENGINE_INTERP):
        progs = [F.compile(w.text, w.k).set_option(L.OPT_ENGINE, engine) for w in mix]
        dev = torch.full((len(progs),), -1, dtype=torch.int64, device="cuda")
        F.count_each(progs, dev)
        torch.cuda.synchronize()
        assert F.read_counts(dev) == want
        F.count_each(progs, dev)            # again: the self-resetting counters start from zero
        torch.cuda.synchronize()
        assert F.read_counts(dev) == want
