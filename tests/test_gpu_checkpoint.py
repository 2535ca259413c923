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


@pytest.mark.parametrize("wl", [W.TRANSITIVE6, W.TRIFREE9, W.AUT6, W.posets(5)], ids=lambda w: w.family)
def test_scheduled_counts_unchanged(wl):
    """fbg_schedule_units reorders the items, longest measured first; counts,
    unit ranges and per-unit counts stay the same, and an option change drops
    the order."""
    import torch
    p = F.compile(wl.text, wl.k)
    want = p.count()
    _, nunits = p.unit_vars()
    per_unit = torch.zeros(nunits, dtype=torch.int64, device="cuda")
    p.count_units(per_unit)
    p.schedule_units()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(3):
        p.count_async(out)
        assert int(out.item()) == want
    assert p.count() == want
    assert p.count_range(0, nunits // 2) + p.count_range(nunits // 2, nunits) == want
    again = torch.zeros_like(per_unit)
    p.count_units(again)
    assert torch.equal(again, per_unit)
    tr = torch.zeros(2 * nunits, dtype=torch.int64, device="cuda")
    p.debug_unit_trace(tr)
    t = tr.cpu().view(-1, 2)
    assert int(t[:, 0].sum()) > 0 and int(t[:, 1].min()) >= 0
    p.set_option(L.OPT_MIN_BLOCKS, 1)
    assert p.count() == want


def test_counts_interleaved_with_tables_and_model_lists():
    """Plain counts reset their own counters; tables, model lists, unit
    counts, statistics and ranges in between must not disturb them."""
    import numpy as np
    import torch
    import oracle
    wl = W.posets(5)
    th = oracle.Theory(wl.text, wl.k)
    want = th.count()
    p = F.compile(wl.text, wl.k)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    words = torch.zeros(p.table_words(), dtype=torch.int64, device="cuda")
    models = torch.zeros(8192, dtype=torch.int64, device="cuda")
    _, nunits = p.unit_vars()
    per_unit = torch.zeros(nunits, dtype=torch.int64, device="cuda")
    for r in range(3):
        assert p.count() == want
        p.truth_table(words)
        p.count_async(out)
        assert int(out.item()) == want
        assert p.enumerate_models(models) == (want, want)
        assert p.count() == want
        p.count_units(per_unit)
        assert int(per_unit.sum()) == want
        p.count_async(out)
        p.count_async(out)
        assert int(out.item()) == want
        assert p.count_range(0, nunits // 3) + p.count_range(nunits // 3, nunits) == want
        p.set_option(L.OPT_STATS, 1)
        assert p.count() == want
        p.set_option(L.OPT_STATS, 0)
        assert p.count() == want
    assert np.array_equal(words.cpu().numpy().view(np.uint64), th.table())


def test_item_trace_covers_every_item():
    """fbg_debug_item_trace times each (unit, warp slice) item of a natural
    launch; the wrong buffer size is refused."""
    import torch
    p = F.compile(W.TRIFREE9.text, 9)
    want = p.count()
    lay = p.debug_dump(0)["layout"]
    _, nunits = p.unit_vars()
    nitems = nunits << lay["warp_bits"]
    ns = torch.zeros(nitems, dtype=torch.int64, device="cuda")
    p.debug_item_trace(ns)
    t = ns.cpu()
    # every item is timed (the timer's resolution may round the shortest to 0)
    assert int(t.sum()) > 0 and int((t > 0).sum()) * 2 >= nitems and int((t >= 0).sum()) == nitems
    assert p.count() == want
    with pytest.raises(L.FbgError):
        p.debug_item_trace(torch.zeros(nitems + 1, dtype=torch.int64, device="cuda"))


@pytest.mark.parametrize("wl,opts,want", [
    (W.posets(5), {L.OPT_UNIT_BITS: 2}, 4231),
    (W.posets(5), {L.OPT_UNIT_BITS: 0, L.OPT_LOOP_LEVEL_BITS: 3}, 4231),
    (W.TRANSITIVE6, {}, 9415189),
    (W.TRIFREE9, {}, 246348115),
], ids=["posets5_u2", "posets5_u0", "transitive6", "trifree9"])
def test_split_items_keep_counts(wl, opts, want):
    """fbg_schedule_units hands long items out as pieces over the first loop
    level; counts equal the known counts with and without pieces."""
    import torch
    p = F.compile(wl.text, wl.k)
    for k, v in opts.items():
        p.set_option(k, v)
    p.set_option(L.OPT_SPLIT_ITEMS, 1)
    d = p.debug_dump(0)
    lay = d["layout"]
    assert lay["split_bits"] > 0
    items = (1 << lay["unit_bits"]) << lay["warp_bits"]
    live = len(d["alive_items"]) if "alive_items" in d else items
    assert p.count() == want
    p.schedule_units()
    split = p.debug_dump(0)["item_list_entries"]
    assert split >= live
    assert split <= live << lay["split_bits"]
    if items < 1000:   # fewer items than warps: every item the timer saw is split
        assert split > live
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for _ in range(3):
        p.count_async(out)
        assert int(out.item()) == want
    assert p.count() == want
    p.set_option(L.OPT_SPLIT_ITEMS, 0)
    p.schedule_units()
    assert p.debug_dump(0)["item_list_entries"] == live
    assert p.count() == want
