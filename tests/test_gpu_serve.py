"""GPU: the continuous-batching server (fbg_server_*).  Every result must be
the same alone and in the mix, and equal to the oracle's (exact integers:
bit-exact): whole counts and model lists where the oracle evaluates every
assignment, per-unit subcube counts and sampled model checks above that
(tests/oracle_checks.py)."""
import time

import numpy as np
import pytest

import oracle
import oracle_checks as OC
from oracle import counters as C
import paper_1310_6978_b300 as F
from paper_1310_6978_b300 import _lib as L
from paper_1310_6978_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def mixed_requests(count, seed, n_hi=30):
    reqs = W.request_stream(count, rate_per_s=1e6, seed=seed, n_lo=8, n_hi=n_hi, enum_frac=0.25, cap=1000)
    return [(r.workload, L.MODE_ENUMERATE if r.mode == "enumerate" else L.MODE_COUNT, r.cap) for r in reqs]


def wait_all(srv, ids, timeout=300):
    srv.drain(timeout)
    return {i: srv.poll(i) for i in ids}


def check_with_oracle(wl, mode, cap, r, rng, cache):
    assert r is not None and r["status"] == 0
    OC.check_count(wl, r["count"], rng, cache=cache)
    if mode == L.MODE_ENUMERATE:
        OC.check_models(wl, r["models"], r["count"], cap, rng, cache=cache)


@pytest.mark.parametrize("opts", [{}, {"max_inflight": 3, "tick_units": 16}, {"mem_budget_bytes": 4096}])
def test_results_same_alone_and_in_mix(opts):
    reqs = mixed_requests(60, 21)
    srv = F.Server(**opts)
    ids = [srv.submit(wl.text, wl.k, mode, cap) for wl, mode, cap in reqs]
    res = wait_all(srv, ids)
    rng = np.random.default_rng(21)
    cache = {}
    for i, (wl, mode, cap) in zip(ids, reqs):
        check_with_oracle(wl, mode, cap, res[i], rng, cache)
    # alone: a fresh server, one request at a time; the same result as in the mix
    alone = F.Server(**opts)
    for i, (wl, mode, cap) in list(zip(ids, reqs))[:12]:
        rid = alone.submit(wl.text, wl.k, mode, cap)
        r = wait_all(alone, [rid])[rid]
        assert r["status"] == 0 and r["count"] == res[i]["count"] and r["models"] == res[i]["models"]
    srv.close()
    alone.close()


def test_serving_stream_shape_against_oracle():
    """Requests drawn as the serving benchmark draws them (seed 5: n uniform
    in 16..38, a family with exactly n letters else 3-CNF, 10% model lists
    capped at 10^6), submitted back to back; every count and model list is
    checked against the oracle."""
    reqs = W.request_stream(160, rate_per_s=1e6, seed=5)
    srv = F.Server()
    ids = [srv.submit(r.workload.text, r.workload.k, L.MODE_ENUMERATE if r.mode == "enumerate" else L.MODE_COUNT,
                      r.cap) for r in reqs]
    res = wait_all(srv, ids, timeout=600)
    srv.close()
    rng = np.random.default_rng(5)
    cache = {}
    how = {}
    for i, r in zip(ids, reqs):
        mode = L.MODE_ENUMERATE if r.mode == "enumerate" else L.MODE_COUNT
        check_with_oracle(r.workload, mode, r.cap, res[i], rng, cache)
        how[r.workload.n > 22] = how.get(r.workload.n > 22, 0) + 1
    assert how.get(True, 0) >= 50 and how.get(False, 0) >= 20
    assert max(r.workload.n for r in reqs) == 38


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
    assert res[first]["count"] == C.count_transitive_backtrack(6)
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


def test_completed_queue_hands_out_each_finished_request_once():
    srv = F.Server()
    ids = [srv.submit(W.posets(k).text, k, L.MODE_COUNT, 0) for k in (2, 3, 4, 3)]
    srv.drain(60)
    seen = srv.completed(2) + srv.completed()
    assert sorted(seen) == sorted(ids) and srv.completed() == []
    for rid, want in zip(ids, (3, 19, 219, 19)):
        assert srv.poll(rid)["count"] == want
        srv.release(rid)
    srv.close()


def _wait_programs(srv, want, timeout=180):
    t0 = time.time()
    while srv.stats()["jit_programs"] < want and time.time() - t0 < timeout:
        time.sleep(0.05)
    return srv.stats()["jit_programs"]


def test_recurring_texts_move_to_a_specialised_kernel():
    """Count requests of a text submitted jit_after times (with at least
    jit_min_n letters) are counted by a specialised kernel that a background
    thread compiles; once it is ready, new requests of that text run on it,
    in the same ticks as interpreted requests.  Every count equals the
    oracle's (all points up to n = 22, per-unit subcubes above) and the count
    the interpreter gave the same text before the kernel was ready."""
    fams = [W.triangle_free(7), W.transitive(5), W.posets(5), W.transitive(6)]   # n = 21, 25, 25, 36
    srv = F.Server(jit_min_n=20, jit_after=2)
    first = [srv.submit(wl.text, wl.k) for wl in fams for _ in range(2)]
    srv.drain(300)
    assert _wait_programs(srv, len(fams)) == len(fams)
    before = srv.stats()["jit_requests"]
    others = mixed_requests(24, 33, n_hi=24)
    batch = [(wl, L.MODE_COUNT, 0) for wl in fams for _ in range(3)] + others
    order = np.random.default_rng(3).permutation(len(batch))
    batch = [batch[i] for i in order]
    ids = [srv.submit(wl.text, wl.k, mode, cap) for wl, mode, cap in batch]
    res = wait_all(srv, ids + first)
    assert srv.stats()["jit_requests"] - before >= 3 * len(fams)
    rng, cache = np.random.default_rng(5), {}
    for i, (wl, mode, cap) in zip(ids, batch):
        check_with_oracle(wl, mode, cap, res[i], rng, cache)
    by_text = {}
    for i, (wl, mode, cap) in zip(ids, batch):
        if mode == L.MODE_COUNT:
            by_text.setdefault((wl.text, wl.k), set()).add(res[i]["count"])
    for j, i in enumerate(first):
        assert res[i]["status"] == 0
        assert by_text[(fams[j // 2].text, fams[j // 2].k)] == {res[i]["count"]}
    srv.close()


def test_default_server_specialises_n36_and_jit_off_keeps_the_interpreter():
    wl = W.transitive(6)
    on = F.Server()
    ids = [on.submit(wl.text, wl.k) for _ in range(2)]
    on.drain(300)
    assert _wait_programs(on, 1) == 1
    ids += [on.submit(wl.text, wl.k) for _ in range(2)]
    res = wait_all(on, ids)
    assert on.stats()["jit_requests"] == 2
    assert len({res[i]["count"] for i in ids}) == 1 and res[ids[0]]["status"] == 0
    want = res[ids[-1]]["count"]
    OC.check_count(wl, want, np.random.default_rng(6))
    on.close()
    off = F.Server(jit_min_n=-1)
    ids = [off.submit(wl.text, wl.k) for _ in range(3)]
    res = wait_all(off, ids)
    time.sleep(0.5)
    st = off.stats()
    assert st["jit_programs"] == 0 and st["jit_requests"] == 0
    assert {res[i]["count"] for i in ids} == {want}
    off.close()


def test_requests_without_live_units_finish_with_zero():
    """A request whose build leaves no unit (every unit killed by a conjunct
    over unit letters) has no models: the server finishes it at admission,
    alone and among other requests, and the standalone engines agree."""
    wl = W.cnf3(30, 1, 8.0)            # no unit of the server's count layout survives its build
    text, n = wl.text, wl.k
    p = F.compile(text, n)
    assert p.count() == 0
    assert F.compile(text, n).set_option(L.OPT_ENGINE, L.ENGINE_INTERP).count() == 0
    OC.check_count(wl, 0, np.random.default_rng(40))
    srv = F.Server()
    others = mixed_requests(20, 41, n_hi=24)
    ids = [srv.submit(text, n, L.MODE_COUNT), srv.submit(text, n, L.MODE_ENUMERATE, 100)]
    ids += [srv.submit(wl.text, wl.k, mode, cap) for wl, mode, cap in others]
    ids += [srv.submit(text, n, L.MODE_COUNT)]
    res = wait_all(srv, ids, timeout=120)
    for i in (ids[0], ids[1], ids[-1]):
        assert res[i]["status"] == 0 and res[i]["count"] == 0 and res[i]["models"] == []
    rng, cache = np.random.default_rng(41), {}
    for i, (wl, mode, cap) in zip(ids[2:-1], others):
        check_with_oracle(wl, mode, cap, res[i], rng, cache)
    srv.close()
