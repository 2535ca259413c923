"""GPU: truth tables and model lists by unit ranges (fbg_truth_table_range,
fbg_enumerate_models_range), the parts one GPU of several would compute.
The parts of consecutive ranges, in order, must be the whole table and the
whole capped list of the oracle (exact: bit-exact words, equal lists)."""
import numpy as np
import pytest

import oracle
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import shard
from paper_1310_6978_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [W.cnf3(22, 5, 2.0), W.posets(4), W.transitive(4), W.cnf3(20, 8)]
SHAPES = [{}, {L.OPT_UNIT_BITS: 4, L.OPT_REGS_LOG2: 1, L.OPT_WARPS_LOG2: 1}]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _program(wl, shape):
    p = F.compile(wl.text, wl.k)
    for k, v in shape.items():
        p.set_option(k, v)
    return p


@pytest.mark.parametrize("wl", CASES, ids=lambda w: f"{w.family}{w.param}n{w.n}")
@pytest.mark.parametrize("si", range(len(SHAPES)))
def test_table_ranges_make_the_whole_table(wl, si):
    th = oracle.Theory(wl.text, wl.k)
    want = th.table()
    p = _program(wl, SHAPES[si])
    nunits, wpu = p.table_units(1)
    assert nunits * wpu == max(1, (1 << wl.n) >> 6) or nunits == 1
    for world in (1, 2, 3, 7):
        parts = []
        for r in range(world):
            b, e = shard.unit_range(nunits, r, world)
            if e <= b:
                continue
            t = torch.full(((e - b) * wpu,), -1, dtype=torch.int64, device="cuda")
            p.truth_table_range(b, e, t)
            parts.append(t)
        torch.cuda.synchronize()
        got = torch.cat(parts).cpu().numpy().view(np.uint64)
        assert np.array_equal(got, want), world


@pytest.mark.parametrize("wl", CASES, ids=lambda w: f"{w.family}{w.param}n{w.n}")
@pytest.mark.parametrize("cap", [0, 9, 1000, 1 << 20])
def test_model_ranges_make_the_whole_list(wl, cap):
    th = oracle.Theory(wl.text, wl.k)
    want, wtotal = th.models(cap)
    for shape in SHAPES:
        p = _program(wl, shape)
        nunits, _ = p.table_units(2)
        for world in (2, 5):
            totals, writtens, bufs = [], [], []
            for r in range(world):
                b, e = shard.unit_range(nunits, r, world)
                buf = torch.full((max(1, cap),), -1, dtype=torch.int64, device="cuda")
                t, w = p.enumerate_models_range(b, e, buf, cap) if e > b else (0, 0)
                totals.append(t)
                writtens.append(w)
                bufs.append(buf)
            offsets, keep = shard.keep_counts(totals, writtens, cap)
            merged = np.concatenate([bf[:k].cpu().numpy().view(np.uint64) for bf, k in zip(bufs, keep)])
            assert sum(totals) == wtotal
            assert np.array_equal(merged, want)


def test_range_errors():
    p = F.compile(W.cnf3(22, 5).text, 22)
    nunits, wpu = p.table_units(1)
    t = torch.zeros(wpu, dtype=torch.int64, device="cuda")
    for b, e, n in ((1, 1, wpu), (0, nunits + 1, wpu), (0, 1, wpu + 1)):
        with pytest.raises(L.FbgError) as ei:
            p.truth_table_range(b, e, t[:n] if n <= wpu else torch.zeros(n, dtype=torch.int64, device="cuda"))
        assert ei.value.status == L.FBG_EINVAL
    q = F.compile(W.cnf3(22, 5).text, 22).set_option(L.OPT_ENGINE, L.ENGINE_INTERP)
    with pytest.raises(L.FbgError) as ei:
        q.table_units(2)
    assert ei.value.status == L.FBG_EINVAL
