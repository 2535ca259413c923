"""One count split across ranks (one process per GPU).

The assignment space is cut by the unit bits (the top of the layout): rank g
of G counts a contiguous range of units with ``fbg_count_range`` and the
partial counts are added with one 8-byte all-reduce, the only exchange the
method has (counts over disjoint sets of assignments add, Sec. 3.2).  Truth
tables and model lists split the same way: rank g evaluates the table words
or the models of its contiguous unit range (fbg_truth_table_range,
fbg_enumerate_models_range), and the whole table or list is the
concatenation of the ranks' parts in rank order.  A capped model list needs
one more 8-byte exchange: every rank's number of models, which fixes where
its part starts and how much of it falls under the cap.
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


def keep_counts(totals, written, cap: int):
    """For a model list split over ranks in rank order: rank g found
    totals[g] models in its range and stored the first written[g]; the global
    list keeps the first ``cap`` models overall.  Returns (offsets, keep):
    rank g's models start at position offsets[g] of the global list, and its
    first keep[g] stored models belong to the list."""
    offsets, keep, at = [], [], 0
    for t, w in zip(totals, written):
        offsets.append(at)
        keep.append(max(0, min(w, cap - at)))
        at += t
    return offsets, keep


def table_sharded(prog, group=None, stream=None):
    """This rank's part of the truth table: (index of its first 64-bit word
    in the whole table, a tensor of its words).  ``prog`` needs
    ``table_units(1)`` and ``truth_table_range(begin, end, words, stream)``."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    nunits, wpu = prog.table_units(1)
    begin, end = unit_range(nunits, rank, world)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    words = torch.empty(max(0, end - begin) * wpu, dtype=torch.int64, device=dev)
    if end > begin:
        prog.truth_table_range(begin, end, words, stream)
    return begin * wpu, words


def models_sharded(prog, cap: int, group=None, stream=None):
    """This rank's part of the list of the first ``cap`` models in ascending
    order: (exact number of models over all ranks, position of this rank's
    part in the global list, a tensor of its models that belong to the
    list).  One 8-byte exchange (every rank's model count) sizes the parts.
    ``prog`` needs ``table_units(2)`` and ``enumerate_models_range``."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    nunits, _ = prog.table_units(2)
    begin, end = unit_range(nunits, rank, world)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    buf = torch.empty(max(1, cap), dtype=torch.int64, device=dev)
    total, written = prog.enumerate_models_range(begin, end, buf, cap, stream) if end > begin else (0, 0)
    mine = torch.tensor([to_int64_bits(total), to_int64_bits(written)], dtype=torch.int64, device=dev)
    every = [torch.zeros_like(mine) for _ in range(world)]
    dist.all_gather(every, mine, group=group)
    totals = [int(t[0].item()) & MASK64 for t in every]
    writtens = [int(t[1].item()) & MASK64 for t in every]
    offsets, keep = keep_counts(totals, writtens, cap)
    return sum(totals), offsets[rank], buf[:keep[rank]]
