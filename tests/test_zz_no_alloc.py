"""fbg_count_noalloc: counting without any device allocation by the library.

Callers that cannot let a library call cudaMalloc (a process whose caching
allocator already holds the free device memory, or code held to a fixed,
pre-reserved budget) use this entry point: its scratch -- work counters,
program descriptor, bytecode, constants and work queue -- is one fixed-size
device array compiled into the library.  Its counts must equal the normal
entry point's (fbg_count), exactly, on two calls in a row: the array keeps
the previous call's contents, so each call has to clear what must start at
zero.  Programs too large for the array are refused with FBG_ETOOBIG.

This file is named so that pytest collects it last.
"""
import itertools

import pytest

import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [W.POSET3, W.posets(4), W.equivalences(5), W.transitive(5), W.triangle_free(7), W.automorphisms(5, 7),
         W.cnf3(20, 4), W.cnf3(26, 9), W.BAEQU4, W.TRANSITIVE6]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("wl", CASES, ids=lambda w: f"{w.family}{w.param}n{w.n}")
def test_noalloc_count_equals_fbg_count_twice(wl):
    p = F.compile(wl.text, wl.k)
    want = p.count()                       # the existing entry point
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    for _ in range(2):                     # the array keeps the previous call's contents
        out.fill_(-1)
        p.count_noalloc(out)
        assert int(out.item()) == want


def test_noalloc_on_caller_stream_and_other_programs_between():
    s = torch.cuda.Stream()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    a = F.compile(W.posets(5).text, 5)
    b = F.compile(W.cnf3(22, 3).text, 22)
    want_a, want_b = a.count(), b.count()
    with torch.cuda.stream(s):
        a.count_noalloc(out, stream=s)
        assert int(out.item()) == want_a
        b.count_noalloc(out, stream=s)
        assert int(out.item()) == want_b
        a.count_noalloc(out, stream=s)
        assert int(out.item()) == want_a


def test_noalloc_refuses_programs_larger_than_its_array():
    # all 5-literal clauses over 12 letters: about 150 KB of bytecode
    lines = ["var x(S)"]
    for vs in itertools.combinations(range(12, 24), 5):
        for sg in range(32):
            lines.append(" | ".join(("~" if (sg >> t) & 1 else "") + f"x({v})" for t, v in enumerate(vs)))
    p = F.compile("\n".join(lines) + "\n", 24)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(L.FbgError) as ei:
        p.count_noalloc(out)
    assert ei.value.status == L.FBG_ETOOBIG
    assert "at most" in str(ei.value)
    # a call after the refusal still works
    q = F.compile(W.posets(4).text, 4)
    q.count_noalloc(out)
    assert int(out.item()) == 219


def test_noalloc_first_on_fresh_programs_against_known_counts():
    # programs counted only through fbg_count_noalloc (no fbg_count before):
    # posets on 5 points (4231) and equivalence relations on 5 points
    # (the Bell number 52)
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    for text, k, want in ((W.posets(5).text, 5, 4231), (W.equivalences(5).text, 5, 52)):
        p = F.compile(text, k)
        for _ in range(2):
            out.fill_(-1)
            p.count_noalloc(out)
            assert int(out.item()) == want


def test_noalloc_allocates_no_device_memory():
    # after one warm-up call (the per-device set-up), further calls leave
    # the device's free memory exactly as it was
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    progs = [F.compile(W.posets(4).text, 4), F.compile(W.cnf3(22, 5).text, 22), F.compile(W.triangle_free(7).text, 7)]
    progs[0].count_noalloc(out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        for p in progs:
            p.count_noalloc(out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
