"""GPU: the continuous-batching server (fbg_server_*).  Every result must be
the same alone and in the mix, and equal to the single-program entry points
and, at small n, to the oracle (exact integers: bit-exact)."""
import time

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


def reference(wl, mode, cap):
    p = F.compile(wl.text, wl.k)
    if mode == L.MODE_COUNT:
        return p.count(), []
    buf = torch.zeros(max(1, cap), dtype=torch.int64, device="cuda")
    total, written = p.enumerate_models(buf, cap)
    return total, [int(x) for x in buf[:written].cpu().numpy().view(np.uint64)]


def mixed_requests(count, seed, n_hi=30):
    reqs = W.request_stream(count, rate_per_s=1e6, seed=seed, n_lo=8, n_hi=n_hi, enum_frac=0.25, cap=1000)
    return [(r.workload, L.MODE_ENUMERATE if r.mode == "enumerate" else L.MODE_COUNT, r.cap) for r in reqs]


def wait_all(srv, ids, timeout=300):
    srv.drain(timeout)
    return {i: srv.poll(i) for i in ids}


@pytest.mark.parametrize("opts", [{}, {"max_inflight": 3, "tick_units": 16}, {"mem_budget_bytes": 4096}])
def test_results_same_alone_and_in_mix(opts):
    reqs = mixed_requests(60, 21)
    srv = F.Server(**opts)
    ids = [srv.submit(wl.text, wl.k, mode, cap) for wl, mode, cap in reqs]
    res = wait_all(srv, ids)
    for i, (wl, mode, cap) in zip(ids, reqs):
        r = res[i]
        assert r is not None and r["status"] == 0
        want_count, want_models = reference(wl, mode, cap)
        assert r["count"] == want_count
        if mode == L.MODE_ENUMERATE:
            assert r["models"] == want_models
    # alone: a fresh server, one request at a time
    alone = F.Server(**opts)
    for wl, mode, cap in reqs[:12]:
        rid = alone.submit(wl.text, wl.k, mode, cap)
        r = wait_all(alone, [rid])[rid]
        want_count, want_models = reference(wl, mode, cap)
        assert r["count"] == want_count and (mode == L.MODE_COUNT or r["models"] == want_models)
    srv.close()
    alone.close()


def test_small_requests_equal_oracle_and_latency_fields():
    reqs = mixed_requests(40, 5, n_hi=18)
    srv = F.Server()
    ids = [srv.submit(wl.text, wl.k, mode, cap) for wl, mode, cap in reqs]
    res = wait_all(srv, ids)
    for i, (wl, mode, cap) in zip(ids, reqs):
        th = oracle.Theory(wl.text, wl.k)
        r = res[i]
        assert r["count"] == th.count()
        if mode == L.MODE_ENUMERATE:
            om, _ = th.models(cap)
            assert r["models"] == [int(x) for x in om]
        assert r["submit_s"] <= r["admit_s"] <= r["done_s"]
    st = srv.stats()
    assert st["ticks"] >= 1 and st["launches"] >= 1
    srv.close()


def test_requests_arriving_while_running_join_later_ticks():
    srv = F.Server(tick_units=64)
    big = W.TRANSITIVE6
    first = srv.submit(big.text, big.k, L.MODE_COUNT, 0)
    time.sleep(0.01)
    later = [srv.submit(W.posets(4).text, 4, L.MODE_COUNT, 0) for _ in range(5)]
    res = wait_all(srv, [first] + later)
    assert res[first]["count"] == F.compile(big.text, big.k).count()
    assert all(res[i]["count"] == 219 for i in later)
    srv.close()


def test_submit_errors_and_release():
    srv = F.Server()
    with pytest.raises(L.FbgError) as ei:
        srv.submit("var x\nx &\n", 1)
    assert ei.value.status == L.FBG_EPARSE
    rid = srv.submit(W.POSET3.text, 3)
    srv.drain(60)
    assert srv.poll(rid)["count"] == 19
    srv.release(rid)
    with pytest.raises(L.FbgError):
        srv.poll(rid)
    srv.close()
