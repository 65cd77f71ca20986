"""The region-ordered first pass against the oracle and against the direct kernels.

Forced on small filters (64 regions of a 2^20-bit filter, 4 of a 256-bit one), every
round's records go through the buckets: the junctions must equal the oracle's element
by element, the last round's C_temp must equal the oracle's first pass over that
round's class bit for bit (the same filter, applied in another order), and the
counts must equal those of the direct kernels. For k <= 27 (and not the partially
compacted graph) pass 2 runs on the same records, with one part of the table per
filter region. A round whose records do not fit (a homopolymer puts most positions
into one class) takes the direct kernels, and the other rounds stay ordered.
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


def _eq(got, want):
    assert len(got) == len(want)
    for t, (g, w) in enumerate(zip(got, want)):
        g = np.asarray(g, np.uint64)
        w = np.asarray(w, np.uint64)
        assert np.array_equal(g, w), f"string {t}: {g.size} vs {w.size} junctions"


@functools.lru_cache(maxsize=None)
def _input(split=False):
    seqs = list(G.named_set("plain_single", 0.05))
    seqs += G.random_strings(77, 40, 0, 400)         # short strings, some shorter than k
    seqs += [np.frombuffer(b"ACGT" * 50, np.uint8)]  # a tandem repeat
    if split:
        seqs = G.plant_n_runs(5, seqs)
    return G.concat(seqs)


def _marks(run, m):
    words = run.state(T().STATE_CANDIDATES, (m + 31) // 32)
    return np.unpackbits(words.view(np.uint8), bitorder="little")[:m]


CASES = [
    (25, 1 << 20, 4, 4, {}),
    (31, 1 << 22, 3, 3, {}),
    (63, 1 << 20, 6, 2, {}),
    (15, 1 << 16, 1, 16, {}),
    (12, 1 << 14, 5, 8, {}),
    (25, 1 << 18, 4, 4, {"both_strands": False}),
    (21, 1 << 20, 4, 4, {"split_at_n": True}),
    (25, 1 << 20, 4, 3, {"partial": True}),
    (25, 256, 2, 2, {}),  # four one-word regions; every position survives the first pass
    (25, 1 << 20, 4, 4, {"wide_layout": 1}),  # 64-bit candidate records
]


def _run(bases, off, k, bits, rounds, opts, cut=None):
    """A run over every round with the given class cut (a CUDA tensor), or with the one
    it computes (the cut counts distinct k-mers through the filter, so on a small filter
    it can differ from run to run)."""
    run = T().DeviceBuild(bases, off, k, bits, rounds, opts)
    run.shard_begin(compute_cut=cut is None)
    run.shard_rounds(0, 1, class_cut=cut)
    run.write_output()
    return run


@pytest.mark.parametrize("k,bits,h,rounds,extra", CASES)
def test_ordered_first_pass_matches_oracle_and_direct(k, bits, h, rounds, extra):
    split = extra.get("split_at_n", False)
    both = extra.get("both_strands", True)
    bases, off = _input(split)
    m = int(off[-1])
    q = 256
    base = dict(hashes=h, partition_bins=q, **extra)
    a = _run(bases, off, k, bits, rounds, T().Options(ordered_first_pass=2, **base))
    cut = a.state_tensor(T().STATE_CUTS)
    b = _run(bases, off, k, bits, rounds, T().Options(ordered_first_pass=1, **base), cut)
    assert b.ws_bytes > a.ws_bytes
    sa, sb = a.stats(), b.stats()
    assert sa["ordered_rounds"] == 0 and sb["ordered_rounds"] == rounds
    for key in ("positions", "pass1_marks", "pass2_marks"):
        assert sa[key] == sb[key], key
    _eq(b.result(), a.result())
    if extra.get("partial"):
        return
    _eq(b.result(), O.junctions((bases, off), k, both_strands=both, split_n=split))
    # the last round's C_temp: the oracle's first pass over that round's class
    cuts = b.state(T().STATE_CUTS, rounds + 1)
    marks, _, _, kept = O.pass1_marks((bases, off), k, bits, h, both_strands=both, q=q,
                                      bin_lo=int(cuts[rounds - 1]), bin_hi=int(cuts[rounds]),
                                      split_n=split)
    assert np.array_equal(_marks(b, m), marks)
    assert np.array_equal(_marks(a, m), marks)


def test_a_round_that_does_not_fit_takes_the_direct_kernels():
    """A 200 kbp homopolymer: its one k-mer puts 200 k positions into one class, beyond
    a round's records; that round runs direct, the others ordered, and the output is
    the oracle's."""
    seqs = list(G.named_set("plain_single", 0.05)) + [np.frombuffer(b"A" * 200_000, np.uint8)]
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, 25, 1 << 20, 4,
                          T().Options(hashes=4, partition_bins=256, ordered_first_pass=1))
    run.run()
    st = run.stats()
    assert st["ordered_rounds"] == 3
    _eq(run.result(), O.junctions((bases, off), 25))


def test_ordered_run_repeats_and_replays():
    """The same workspace run twice and a captured plan replayed: identical output (the
    buckets' fill counters, tickets and decision bits start over every round)."""
    bases, off = _input()
    opts = T().Options(hashes=4, partition_bins=256, ordered_first_pass=1)
    run = T().DeviceBuild(bases, off, 25, 1 << 20, 4, opts)
    run.run()
    first = run.result()
    run.run()
    _eq(run.result(), first)
    _eq(first, O.junctions((bases, off), 25))
    run.capture()
    for _ in range(2):
        run.run()
        _eq(run.result(), first)
    assert run.stats()["ordered_rounds"] == 4
    run.release_plan()


def test_fused_table_overflow_is_reported_and_recovered():
    """Pass 2 on the records with a table of 4 regions x 1024 slots: a saturated filter keeps
    every k-mer, which overflows the regions; the run reports it and the host build grows
    the table and runs again."""
    bases, off = _input()
    opts = T().Options(hashes=2, partition_bins=256, ordered_first_pass=1, table_slots=4096)
    run = T().DeviceBuild(bases, off, 25, 256, 2, opts)
    run.run()
    st = run.stats(check=False)
    assert st["rc"] == T().EOVERFLOW and st["overflow"] and st["ordered_rounds"] == 2
    seqs = [bases[int(off[t]):int(off[t + 1])] for t in range(len(off) - 1)]
    got, st = T().twopaco_build_ex(seqs, 25, 256, 2, opts)  # grows the table and reruns
    _eq(got, O.junctions((bases, off), 25))
    assert st["table_slots"] > 4096
