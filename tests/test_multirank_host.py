"""The N > 1 host logic with two gloo ranks on the CPU: max-over-ranks timing
and whole-job throughput of bench.py (replicas), and one count sharded over
the ranks by unit ranges with a single sum (paper_1310_6978_b300.shard).
The per-unit counts come from the oracle here, so no GPU is involved."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleUnits:
    """A program stand-in: units are the values of the top u free letters;
    count_range sums oracle cube counts."""

    def __init__(self, text, k, u):
        import oracle
        self.th = oracle.Theory(text, k)
        self.u = u

    def unit_vars(self):
        n = self.th.n
        return list(range(n - self.u, n)), 1 << self.u

    def count_range(self, begin, end, stream=None):
        n = self.th.n
        mask = ((1 << self.u) - 1) << (n - self.u)
        return sum(self.th.count_cube(mask, unit << (n - self.u)) for unit in range(begin, end))


class HugeCounts:
    """A program stand-in whose units hold 2^63 / nunits models each: the
    sharded sum must reach 2^63, which a signed 64-bit read would turn
    negative."""

    def unit_vars(self):
        return list(range(32)), 1 << 32

    def count_range(self, begin, end, stream=None):
        return (end - begin) << 31


class OracleRanges:
    """A program stand-in for tables and model lists: units are the values of
    the top u letters (each unit a contiguous range of assignment integers);
    the words and models of a unit range come from the oracle."""

    def __init__(self, text, k, u):
        import oracle
        self.th = oracle.Theory(text, k)
        self.u = u

    def table_units(self, mode):
        below = self.th.n - self.u
        return 1 << self.u, max(1, 1 << (below - 6))

    def truth_table_range(self, begin, end, words, stream=None):
        import ctypes
        import numpy as np
        below = self.th.n - self.u
        lo, hi = begin << below, end << below
        buf = np.zeros((hi - lo) >> 6, dtype=np.uint64)
        out = ctypes.c_uint64()
        self.th._lib.oracle_range(self.th._h, lo, hi, ctypes.byref(out), buf.ctypes.data_as(ctypes.c_void_p),
                                  None, 0, None)
        words.copy_(__import__("torch").from_numpy(buf.view(np.int64)))

    def enumerate_models_range(self, begin, end, buf, cap, stream=None):
        import numpy as np
        import torch
        below = self.th.n - self.u
        models, total = self.th.models(cap, begin << below, end << below)
        buf[:len(models)] = torch.from_numpy(np.asarray(models, dtype=np.uint64).view(np.int64))
        return total, len(models)


def worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1310_6978_b300 import shard
        from paper_1310_6978_b300 import workloads as W
        t_max = bench.max_over_ranks(1.0 + rank, world, "cpu")
        rate = bench.whole_job_rate(world * 10 ** 9, t_max)
        wl = W.posets(4)
        total = shard.count_sharded(OracleUnits(wl.text, wl.k, 5))
        huge = shard.count_sharded(HugeCounts())
        # tables and model lists: every rank's part, gathered in rank order
        rp = OracleRanges(wl.text, wl.k, 3)
        first, words = shard.table_sharded(rp)
        tables = [None] * world
        dist.all_gather_object(tables, (first, words.numpy().view("uint64").tolist()))
        lists = {}
        for cap in (0, 7, 100, 1000):
            mtotal, offset, models = shard.models_sharded(rp, cap)
            parts = [None] * world
            dist.all_gather_object(parts, (offset, models.numpy().view("uint64").tolist()))
            lists[cap] = (mtotal, parts)
        dist.barrier()
        q.put((rank, t_max, rate, total, huge, tables, lists))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_two_and_three_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    import numpy as np
    import oracle
    from paper_1310_6978_b300 import workloads as W
    th = oracle.Theory(W.posets(4).text, 4)
    full = [int(x) for x in th.table()]
    for rank, t_max, rate, total, huge, tables, lists in res:
        # the table parts, in rank order, are the whole table
        got, at = [], 0
        for first, words in tables:
            assert first == at
            got += words
            at += len(words)
        assert got == full
        for cap, (mtotal, parts) in lists.items():
            want, wtotal = th.models(cap)
            assert mtotal == wtotal == 219
            merged = []
            for offset, models in parts:
                assert offset == len(merged) or not models
                merged += models
            assert merged == [int(x) for x in want]
        assert huge == 1 << 63                        # a tautology at n = 63, summed unsigned
        assert t_max == float(world)                  # the slowest rank: 1 + (world - 1)
        assert rate == pytest.approx(world / t_max)   # world * 1e9 units over t_max, in G/s
        assert total == 219                           # posets on 4 points, summed over the slices


def test_unit_ranges_cover_once():
    from paper_1310_6978_b300.shard import unit_range
    for nunits in (1, 2, 7, 8192):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                b, e = unit_range(nunits, r, world)
                assert 0 <= b <= e <= nunits
                seen += range(b, e)
            assert seen == list(range(nunits))
    with pytest.raises(ValueError):
        unit_range(8, 2, 2)


def test_keep_counts_cut_the_list_at_the_cap():
    from paper_1310_6978_b300.shard import keep_counts
    assert keep_counts([3, 0, 5, 2], [3, 0, 5, 2], 6) == ([0, 3, 3, 8], [3, 0, 3, 0])
    assert keep_counts([3, 4], [3, 4], 100) == ([0, 3], [3, 4])
    assert keep_counts([10, 4], [2, 2], 2) == ([0, 10], [2, 0])   # a rank stores at most cap
    assert keep_counts([], [], 5) == ([], [])


def test_int64_bit_patterns_of_counts():
    from paper_1310_6978_b300.shard import MASK64, to_int64_bits
    for c in (0, 1, (1 << 63) - 1, 1 << 63, MASK64):
        assert to_int64_bits(c) & MASK64 == c
        assert -(1 << 63) <= to_int64_bits(c) < (1 << 63)
    with pytest.raises(ValueError):
        to_int64_bits(-1)
