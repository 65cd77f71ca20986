"""The partially compacted graph (Discussion section: the second pass omitted) on the GPU.

With options.partial the output positions are the first pass's survivors of
every round -- C_temp of each class, united -- and the edges join consecutive
output positions. Both are compared element by element with the oracle's
restatement of the same first pass (oracle_pass1, run per class with the cut
the GPU chose) and with its edges over those flags. Integer work: exact.
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
def _input(scale, split):
    seqs = G.named_set("plain_single", scale)
    if split:
        seqs = G.plant_n_runs(4, seqs)
    return G.concat(seqs)


def _oracle_partial(bases, off, k, bits, h, both, split, rounds, cuts, q):
    """Union over the classes of the first pass's marks, one fresh filter per class."""
    m = int(off[-1])
    union = np.zeros(m, np.uint8)
    for r in range(rounds):
        lo, hi = (0, 1) if rounds == 1 else (int(cuts[r]), int(cuts[r + 1]))
        marks, _, _, _ = O.pass1_marks((bases, off), k, bits, h, both_strands=both,
                                       q=1 if rounds == 1 else q, bin_lo=lo, bin_hi=hi,
                                       split_n=split)
        assert not np.any(union & marks)
        union |= marks
    return union


@pytest.mark.parametrize("k,bits,h,both,split,rounds,wide", [
    (25, 1 << 18, 4, True, False, 1, 0),
    (25, 1 << 16, 3, True, False, 3, 0),
    (31, 1 << 18, 4, False, False, 1, 0),
    (63, 1 << 18, 5, True, False, 2, 0),
    (100, 1 << 18, 4, True, False, 2, 0),
    (21, 1 << 17, 4, True, True, 2, 0),
    (25, 1 << 17, 4, True, False, 2, 1),
])
def test_partial_output_is_the_first_pass_survivors(k, bits, h, both, split, rounds, wide):
    bases, off = _input(0.05, split)
    q = 256
    opts = T().Options(hashes=h, both_strands=both, split_at_n=split, partition_bins=q,
                       wide_layout=wide, partial=True)
    run = T().DeviceBuild(bases, off, k, bits, rounds, opts)
    run.run()
    got = run.result()
    st = run.stats()
    cuts = run.state(T().STATE_CUTS, rounds + 1) if rounds > 1 else None
    want = _oracle_partial(bases, off, k, bits, h, both, split, rounds, cuts, q)
    for t, g in enumerate(got):
        w = np.flatnonzero(want[int(off[t]):int(off[t + 1])]).astype(np.uint64)
        assert np.array_equal(np.asarray(g, np.uint64), w), t
    assert st["pass2_marks"] == st["pass1_marks"] == int(want.sum())
    # every junction is still there, and the filter left false candidates to compact
    flags, _, _ = O.junction_flags((bases, off), k, both_strands=both, split_n=split)
    assert np.all(want >= flags) and int(want.sum()) > int(flags.sum())


def test_partial_edges_match_oracle():
    bases, off = _input(0.05, False)
    seqs = [bases[int(off[t]):int(off[t + 1])] for t in range(len(off) - 1)]
    k, bits, h = 25, 1 << 17, 3
    ctx = T().Context()
    ctx.build(seqs, k, bits, 1, T().Options(hashes=h, partial=True))
    eoff, got = ctx.edges()
    ctx.close()
    marks, _, _, _ = O.pass1_marks((bases, off), k, bits, h)
    want = O.edges((bases, off), k, flags=marks)
    assert np.array_equal(np.diff(eoff), want["per_string"])
    for f in ("from_hi", "from_lo", "to_hi", "to_lo", "start", "length", "from_rc", "to_rc"):
        assert np.array_equal(got[f].astype(np.uint64), want[f].astype(np.uint64)), f


def test_partial_run_launches_no_second_pass():
    bases, off = _input(0.02, False)
    full = T().DeviceBuild(bases, off, 25, 1 << 18, 1, T().Options(hashes=4))
    part = T().DeviceBuild(bases, off, 25, 1 << 18, 1, T().Options(hashes=4, partial=True))
    assert part.ws_bytes < full.ws_bytes
    n0 = T().twopaco_kernel_launches()
    full.run()
    n1 = T().twopaco_kernel_launches()
    part.run()
    n2 = T().twopaco_kernel_launches()
    assert (n1 - n0) - (n2 - n1) == 4  # table setup, table clear, pass-2 insert and classify
    a, b = full.result(), part.result()
    for x, y in zip(a, b):
        assert np.all(np.isin(x, y))  # the junctions are among the partial positions
