"""The large-input workspace layout on small inputs, against the oracle.

Inputs of 2^31 bases and more keep 64-bit candidate records and no probe
descriptors, and tables of 2^32 slots and more keep no slot per candidate; the
``wide_layout`` option selects those layouts at any size, so that the same
bit-exact checks as elsewhere (junction positions, the pass-1 candidate
bitmap, edges) cover them.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_1602_05856_gb300 import genomes as G
from tests import brute

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05856_gb300 import build
    build.build()
    from paper_1602_05856_gb300 import twopaco
    twopaco.load()


def T():
    from paper_1602_05856_gb300 import twopaco
    return twopaco


def _eq(got, want):
    assert len(got) == len(want)
    for t, (g, w) in enumerate(zip(got, want)):
        g = np.asarray(g, dtype=np.uint64)
        w = np.asarray(w, dtype=np.uint64)
        assert np.array_equal(g, w), (t, g.size, w.size, np.setdiff1d(g, w)[:8], np.setdiff1d(w, g)[:8])


def _bits_to_marks(words, m):
    b = np.unpackbits(np.asarray(words, dtype=np.uint32).view(np.uint8), bitorder="little")
    return b[:m]


@functools.lru_cache(maxsize=None)
def _random_set(k):
    rng = np.random.default_rng(7000 + k)
    seqs = [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 6, 0, 3000, b"ACGT")]
    seqs += [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 3, 50, 700, b"AC")]
    seqs.append(brute.revcomp(seqs[0]))
    seqs.append(seqs[1][100:900] + seqs[2][:400])
    seqs.append("A" * (k + 5))
    return seqs


@pytest.mark.parametrize("wide", [1, 2])
@pytest.mark.parametrize("k,both", [(5, True), (25, True), (31, False), (47, True), (63, True),
                                    (100, True)])
def test_random_inputs_match_oracle(wide, k, both):
    seqs = _random_set(k)
    want = O.junctions(seqs, k, both_strands=both)
    for bits, h, rounds in ((256, 1, 1), (1 << 12, 3, 1), (1 << 18, 4, 1), (1 << 14, 4, 3)):
        got, _ = T().twopaco_build_ex(seqs, k, bits, rounds,
                                      T().Options(hashes=h, both_strands=both, partition_bins=64,
                                                  wide_layout=wide))
        _eq(got, want)


@pytest.mark.parametrize("wide", [1, 2])
@pytest.mark.parametrize("k,bits,h", [(25, 1 << 20, 3), (31, 1 << 18, 4), (63, 1 << 16, 5)])
def test_pass1_candidates_and_counts(wide, k, bits, h):
    """The candidate bitmap and the pass counters do not depend on the layout."""
    bases, off = G.concat(G.named_set("plain_single", 0.1))
    m = int(off[-1])
    run = T().DeviceBuild(bases, off, k, bits, 1, T().Options(hashes=h, wide_layout=wide))
    run.run()
    got = run.result()
    st = run.stats()
    ctemp = _bits_to_marks(run.state(T().STATE_CANDIDATES, (m + 31) // 32), m)
    marks, _, active, kept = O.pass1_marks((bases, off), k, bits, h)
    assert np.array_equal(ctemp, marks)
    assert st["pass1_marks"] == kept and st["positions"] == active
    _eq(got, O.junctions((bases, off), k))


@pytest.mark.parametrize("wide", [1, 2])
def test_rounds_and_list_overflow(wide):
    seqs = G.named_set("plain_single", 0.1)
    bases, off = G.concat(seqs)
    want = O.junctions((bases, off), 25)
    for bits, h, rounds, recs in ((1 << 22, 4, 4, 0), (1 << 20, 3, 1, 1000), (1 << 18, 2, 3, 500)):
        got, _ = T().twopaco_build_ex(seqs, 25, bits, rounds,
                                      T().Options(hashes=h, partition_bins=256, candidate_records=recs,
                                                  wide_layout=wide))
        _eq(got, want)


@pytest.mark.parametrize("wide", [1, 2])
def test_split_n_and_edges(wide):
    rng = np.random.default_rng(31)
    base = [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 5, 0, 2000, b"ACGT")]
    seqs = []
    for s in base:
        s = bytearray(s.encode())
        for _ in range(3):
            a = int(rng.integers(0, len(s) + 1))
            s[a:a] = b"N" * int(rng.integers(1, 40))
        seqs.append(s.decode())
    opts = T().Options(hashes=3, split_at_n=True, wide_layout=wide)
    got, _ = T().twopaco_build_ex(seqs, 25, 1 << 16, 2, opts)
    _eq(got, O.junctions(seqs, 25, split_n=True))
    ctx = T().Context()
    try:
        ctx.build(seqs, 25, 1 << 16, 1, opts)
        off, got = ctx.edges()
        want = O.edges(seqs, 25, split_n=True)
        assert np.array_equal(np.diff(off), want["per_string"])
        for f in ("from_hi", "from_lo", "to_hi", "to_lo", "start", "length", "from_rc", "to_rc"):
            assert np.array_equal(got[f].astype(np.uint64), want[f].astype(np.uint64)), f
    finally:
        ctx.close()
