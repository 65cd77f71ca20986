"""One build split over several GPUs by k-mer class (one process per GPU).

Algorithm 3 (section "Multiple Rounds") splits the k-mers into classes and
runs one round per class; every position belongs to exactly one class, a
round decides only its own class's positions, and C_final is the union of the
rounds' results, which are disjoint. So the rounds can run on different GPUs
over the same input with a single exchange at the end. Rank g of G:

1. packs its own copy of the input (``twopaco_shard_begin``); rank 0 also
   counts the partition bins and cuts the classes;
2. receives rank 0's cut (a broadcast of rounds + 1 words into its workspace);
3. runs the rounds r with r % G == g (``twopaco_shard_rounds``);
4. merges the C_final bitmaps with one all-reduce of their 32-bit words: the
   bitmaps are disjoint, so their integer sum is their bitwise OR (no carry
   can occur), which any backend's SUM computes;
5. writes the output from the merged C_final (rank 0 only, unless asked).

This module holds the host logic only; the GPU work is the library's. Its
collectives come from ``torch.distributed`` (NCCL between GPUs, gloo in the
CPU tests, where a stand-in run object takes the library's place).
"""
from __future__ import annotations

from typing import List, Sequence

from . import twopaco


def owned_rounds(rank: int, world: int, rounds: int) -> List[int]:
    """The rounds (k-mer classes) rank runs: r with r % world == rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    return list(range(rank, rounds, world))


def merge_disjoint_bitmaps(words, dist) -> None:
    """OR of disjoint bitmaps of 32-bit words across ranks, in place (an all-reduce SUM)."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(words, op=dist.ReduceOp.SUM)


def broadcast_cut(cut, dist) -> None:
    """Rank 0's class cut to every rank, in place."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.broadcast(cut, src=0)


def sharded_build(run, rank: int, world: int, dist=None, write_on: Sequence[int] = (0,)) -> None:
    """Steps 1-5 above on ``run`` (a ``twopaco.DeviceBuild``, or any object with its
    shard_begin / shard_rounds / state_tensor / write_output methods)."""
    run.shard_begin(compute_cut=(rank == 0))
    if run.rounds > 1:
        broadcast_cut(run.state_tensor(twopaco.STATE_CUTS), dist)
    run.shard_rounds(rank, world)
    merge_disjoint_bitmaps(run.state_tensor(twopaco.STATE_JUNCTIONS), dist)
    if rank in write_on:
        run.write_output()
