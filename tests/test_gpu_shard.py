"""A build split by k-mer class, its shards run one after the other on one GPU.

Each shard has its own workspace and its own copy of the packed input, as it
would on its own GPU. The leader cuts the classes; the others take its cut
(passed as a device pointer); each runs its rounds; the C_final bitmaps are
merged by summing their 32-bit words (disjoint bits) into the leader's
workspace, which then writes the output. The junctions must equal the
oracle's, element by element, for any number of shards.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_1602_05856_gb300 import genomes as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05856_gb300 import build
    build.build()


def T():
    from paper_1602_05856_gb300 import twopaco
    return twopaco


@functools.lru_cache(maxsize=None)
def _input(scale=0.1, split=False):
    seqs = G.named_set("plain_single", scale)
    if split:
        seqs = G.plant_n_runs(8, seqs)
    return G.concat(seqs)


def _sharded(bases, off, k, bits, rounds, n_shards, **opt):
    opts = T().Options(hashes=4, partition_bins=256, **opt)
    runs = [T().DeviceBuild(bases, off, k, bits, rounds, opts) for _ in range(n_shards)]
    for g, run in enumerate(runs):
        run.shard_begin(compute_cut=(g == 0))
    cut = runs[0].state_tensor(T().STATE_CUTS)
    for g, run in enumerate(runs):
        run.shard_rounds(g, n_shards, class_cut=None if g == 0 else cut)
    leader = runs[0].state_tensor(T().STATE_JUNCTIONS)
    for run in runs[1:]:
        other = run.state_tensor(T().STATE_JUNCTIONS)
        assert not bool(((leader & other) != 0).any()), "shards share a junction"
        leader += other  # disjoint bits: the sum is the OR
    runs[0].write_output()
    return runs


@pytest.mark.parametrize("k,rounds,n_shards", [(25, 2, 2), (25, 5, 2), (31, 6, 3), (63, 4, 4),
                                               (100, 3, 2), (25, 3, 5)])
def test_shards_merge_to_the_junctions(k, rounds, n_shards):
    bases, off = _input()
    runs = _sharded(bases, off, k, 1 << 20, rounds, n_shards)
    want = O.junctions((bases, off), k)
    got = runs[0].result()
    for g, w in zip(got, want):
        assert np.array_equal(np.asarray(g, np.uint64), w)
    st = [r.stats() for r in runs]
    # each shard counts the junctions of its own rounds; the merged output holds all
    assert sum(s["pass2_marks"] for s in st) == sum(w.size for w in want)
    assert int(runs[0].out_offsets[-1].item()) == sum(w.size for w in want)
    n_pos = sum(max(0, int(off[t + 1] - off[t]) - k + 1) for t in range(len(off) - 1))
    assert all(s["positions"] == n_pos for s in st[:min(n_shards, rounds)])


def test_shards_with_n_splitting():
    bases, off = _input(0.05, split=True)
    runs = _sharded(bases, off, 21, 1 << 18, 4, 2, split_at_n=True)
    want = O.junctions((bases, off), 21, split_n=True)
    for g, w in zip(runs[0].result(), want):
        assert np.array_equal(np.asarray(g, np.uint64), w)


def test_partial_shards_are_the_first_pass_per_class():
    """Without the second pass the merged output is the union of each class's first-pass
    survivors under the leader's cut."""
    bases, off = _input(0.05)
    k, bits, h, rounds, q = 25, 1 << 16, 4, 3, 256
    runs = _sharded(bases, off, k, bits, rounds, 2, partial=True)
    cuts = runs[0].state(T().STATE_CUTS, rounds + 1)
    union = np.zeros(int(off[-1]), np.uint8)
    for r in range(rounds):
        marks, _, _, _ = O.pass1_marks((bases, off), k, bits, h, q=q, bin_lo=int(cuts[r]),
                                       bin_hi=int(cuts[r + 1]))
        union |= marks
    for t, g in enumerate(runs[0].result()):
        assert np.array_equal(np.asarray(g, np.uint64),
                              np.flatnonzero(union[int(off[t]):int(off[t + 1])]).astype(np.uint64))
