"""Reproducible grouped SUM over several ranks (one process per GPU).

Each rank aggregates its own rows into a local state; one exchange then
combines the ranks.  Because a state holds exact integers on a fixed grid,
the merge of two states (operator+=(repro) of Sec. V, Algorithm 4's merge,
equal-window case eq. (2)) gives the same bytes in any order or tree, so the
result does not depend on the number of ranks or on how rows were sharded.

The exchange is a reduce-scatter by group blocks followed by an all-gather of
finalized values:
  1. the G groups are cut into one contiguous block per rank;
  2. all_to_all_single sends block j of every rank's records to rank j;
  3. rank j merges the world copies of its block (rank order, for a fixed
     schedule -- any order gives the same bytes) and finalizes it;
  4. all_gather of the finalized blocks gives every rank the T[G] result.
Per rank this moves about (world-1)/world of one state plus G values, instead
of world-1 whole states for an all-gather of states.

The merge itself is a parameter: on the GPU it is the library's merge kernel
(`device_merge`); any function that merges record arrays in place works, so
the host logic runs on CPU ranks (gloo) too.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Tuple

import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int, align: int = 4) -> Tuple[int, int]:
    """Contiguous rows [lo, hi) of rank `rank`; boundaries are multiples of
    `align` rows so every shard keeps the 16-byte alignment of its columns."""
    per = -(-n // world)
    per = -(-per // align) * align
    lo = min(n, rank * per)
    return lo, min(n, lo + per)


def group_blocks(G: int, world: int) -> List[Tuple[int, int]]:
    """One contiguous group range per rank, sizes differing by at most one."""
    base, extra = divmod(G, world)
    out, g0 = [], 0
    for r in range(world):
        g1 = g0 + base + (1 if r < extra else 0)
        out.append((g0, g1))
        g0 = g1
    return out


MergeFn = Callable[[torch.Tensor, torch.Tensor], None]


def reduce_scatter_records(records: torch.Tensor, merge_fn: MergeFn, group=None) -> Tuple[int, int, torch.Tensor]:
    """records: uint8[G, rec] of this rank.  Returns (g0, g1, merged) with
    merged = the merge over all ranks of records[g0:g1], for this rank's
    block [g0, g1)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    G, rec = records.shape
    blocks = group_blocks(G, world)
    B = max(1, max(g1 - g0 for g0, g1 in blocks))
    send = torch.zeros((world, B, rec), dtype=torch.uint8, device=records.device)
    for j, (g0, g1) in enumerate(blocks):
        send[j, : g1 - g0] = records[g0:g1]
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv.view(-1), send.view(-1), group=group)
    g0, g1 = blocks[rank]
    mine = recv[0, : g1 - g0].clone()
    for j in range(1, world):
        if g1 > g0:
            merge_fn(mine, recv[j, : g1 - g0].contiguous())
    return g0, g1, mine


def allgather_blocks(block: torch.Tensor, G: int, group=None) -> torch.Tensor:
    """Concatenate every rank's block of a length-G vector (blocks as in
    group_blocks) into the full vector on every rank."""
    world = dist.get_world_size(group)
    blocks = group_blocks(G, world)
    B = max(1, max(g1 - g0 for g0, g1 in blocks))
    pad = torch.zeros((B,) + tuple(block.shape[1:]), dtype=block.dtype, device=block.device)
    pad[: block.shape[0]] = block
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[j][: g1 - g0] for j, (g0, g1) in enumerate(blocks)])


def max_over_ranks(x: float, group=None, device=None) -> float:
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def or_over_ranks(x: int, group=None, device=None) -> int:
    """Bitwise OR of one integer (an error word) over the ranks."""
    parts = [torch.zeros(1, dtype=torch.int64, device=device) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, torch.tensor([int(x)], dtype=torch.int64, device=device), group=group)
    out = 0
    for p in parts:
        out |= int(p.item())
    return out


# ------------------------------------------------------------ GPU states

def device_merge(dtype, L: int) -> MergeFn:
    """Merge of record arrays in place with the library's record merge kernel
    (repro_merge_records): no state is built around a block, nothing is
    copied.  dtype is unused (records are exact integers)."""
    from . import _check, _stream, lib

    def merge(dst: torch.Tensor, src: torch.Tensor) -> None:
        if not (dst.is_contiguous() and src.is_contiguous()) or dst.shape != src.shape:
            raise ValueError("record blocks must be contiguous and of the same shape")
        g = dst.shape[0]
        _check(lib().repro_merge_records(dst.data_ptr(), src.data_ptr(), L, g, _stream(dst.device)),
               "repro_merge_records")

    return merge


def allreduce_groupby(state, group=None) -> torch.Tensor:
    """Combine every rank's State (same G, L, dtype) and return the finalized
    values.dtype[G] result on every rank; raises ReproError on every rank if
    any rank's state recorded a data error."""
    from . import HEADER_BYTES, ReproError, State

    G, L = state.G, state.L
    rec = (state.tensor.numel() - HEADER_BYTES) // G
    errors = or_over_ranks(state.error_word(), group, device=state.device)
    records = state.tensor[HEADER_BYTES:].view(G, rec)
    g0, g1, mine = reduce_scatter_records(records, device_merge(state.dtype, L), group)
    if g1 > g0:
        blk = State(g1 - g0, L, state.dtype, device=state.device)
        blk.tensor[HEADER_BYTES:].copy_(mine.reshape(-1))
        vals = blk.finalize()
    else:
        vals = torch.empty(0, dtype=state.dtype, device=state.device)
    out = allgather_blocks(vals, G, group)
    status = error_status(errors)
    if status:
        raise ReproError(status, "allreduce_groupby")
    return out


def error_status(word: int) -> int:
    """repro_status for a state error word (REPRO_ERR_KEY, _TIMEOUT, _LAYOUT)."""
    if word & 1:
        return 2
    if word & 2:
        return 6
    if word & 4:
        return 7
    return 0
