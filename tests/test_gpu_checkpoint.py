"""GPU: counts beyond n = 40 and chunked counts with checkpoint/resume."""
import json

import pytest

from oracle import counters as C
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import checkpoint
from paper_1310_6978_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_n49_counts_match_independent_counters():
    # 49 letters: partial orders and equivalence relations on 7 points
    assert F.compile(W.posets(7).text, 7).count() == C.count_posets_c(7) == 6129859
    assert F.compile(W.equivalences(7).text, 7).count() == C.bell(7) == 877


@pytest.mark.parametrize("engine", [L.ENGINE_JIT, L.ENGINE_INTERP])
def test_count_ranges_sum_to_the_count(engine):
    p = F.compile(W.TRANSITIVE6.text, 6).set_option(L.OPT_ENGINE, engine)
    total = p.count()
    _, nunits = p.unit_vars()
    cuts = [0, 1, 7, nunits // 3, nunits // 3 + 1, nunits - 5, nunits]
    parts = [p.count_range(a, b) for a, b in zip(cuts, cuts[1:])]
    assert sum(parts) == total == C.count_transitive_backtrack(6)
    assert p.count_range(5, 5) == 0
    with pytest.raises(L.FbgError):
        p.count_range(9, 3)


def test_resume_after_interruption(tmp_path):
    path = str(tmp_path / "ck.json")
    p = F.compile(W.TRIFREE9.text, 9)
    _, nunits = p.unit_vars()
    st = checkpoint.count_resumable(p, path, chunk_units=nunits // 8, max_chunks=3)
    assert not st["done"] and st["chunks"] == 3
    saved = json.load(open(path))
    assert saved["next_unit"] == 3 * (nunits // 8)
    # a new program object (a restarted process) resumes from the file
    q = F.compile(W.TRIFREE9.text, 9)
    st = checkpoint.count_resumable(q, path, chunk_units=nunits // 8)
    assert st["done"] and st["count"] == C.count_triangle_free_backtrack(9)
    # a checkpoint of another program is refused
    with pytest.raises(ValueError):
        checkpoint.count_resumable(F.compile(W.TRANSITIVE6.text, 6), path)


def test_rank_slices_add_up():
    """The unit slices that count_sharded gives each rank, counted one after
    another on this GPU, add up to the count."""
    from paper_1310_6978_b300.shard import unit_range
    p = F.compile(W.triangle_free(9).text, 9)
    total = p.count()
    _, nunits = p.unit_vars()
    for world in (2, 3, 8):
        assert sum(p.count_range(*unit_range(nunits, r, world)) for r in range(world)) == total
