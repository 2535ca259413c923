"""One count split across ranks (one process per GPU).

The assignment space is cut by the unit bits (the top of the layout): rank g
of G counts a contiguous range of units with ``fbg_count_range`` and the
partial counts are added with one 8-byte all-reduce, the only exchange the
method has (counts over disjoint sets of assignments add, Sec. 3.2).  Truth
tables and model lists would concatenate per-rank slices in rank order; only
the count is provided here.
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1


def to_int64_bits(count: int) -> int:
    """The signed 64-bit integer with the same bits as the unsigned count
    (a torch.int64 element holds it; a count may reach 2^63 at n = 63)."""
    if not 0 <= count <= MASK64:
        raise ValueError("a count is an unsigned 64-bit integer")
    return count - (1 << 64) if count >> 63 else count


def unit_range(nunits: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous slice of [0, nunits) for ``rank``: sizes differ by at most
    one, slices are disjoint and cover every unit in rank order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(nunits, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def count_sharded(prog, group=None, stream=None) -> int:
    """l_{T,n} of ``prog`` with the units shared out over the ranks of
    ``group`` (torch.distributed must be initialised).  ``prog`` needs
    ``unit_vars()`` and ``count_range(begin, end, stream)``; every rank must
    hold the same program.  The sum travels on the GPU for NCCL and on the
    host for gloo."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    _, nunits = prog.unit_vars()
    begin, end = unit_range(nunits, rank, world)
    local = prog.count_range(begin, end, stream) if end > begin else 0
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    # the 64-bit words add modulo 2^64 whatever their sign, so the sum read
    # back as unsigned is the exact count (at most 2^63)
    t = torch.tensor([to_int64_bits(local)], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item()) & MASK64
