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
        dist.barrier()
        q.put((rank, t_max, rate, total, huge))
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
    for rank, t_max, rate, total, huge in res:
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


def test_int64_bit_patterns_of_counts():
    from paper_1310_6978_b300.shard import MASK64, to_int64_bits
    for c in (0, 1, (1 << 63) - 1, 1 << 63, MASK64):
        assert to_int64_bits(c) & MASK64 == c
        assert -(1 << 63) <= to_int64_bits(c) < (1 << 63)
    with pytest.raises(ValueError):
        to_int64_bits(-1)
