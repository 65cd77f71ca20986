"""N splitting on the GPU against the oracle (split_n): an N ends its string.

Bit-exact: junction positions per string, the pass-1 candidate bitmap, and
the compacted-graph edges, on random strings with N runs of every length
around k and on related genomes with assembly-gap-like N runs.
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


def _with_ns(rng, s, k):
    s = bytearray(s.encode() if isinstance(s, str) else bytes(s))
    for _ in range(int(rng.integers(0, 6))):
        a = int(rng.integers(0, len(s) + 1))
        s[a:a] = b"N" * int(rng.integers(1, 2 * k + 3))
    if rng.integers(0, 3) == 0:
        s[:0] = b"n" * int(rng.integers(1, 4))
    if rng.integers(0, 3) == 0:
        s += b"N" * int(rng.integers(1, 4))
    return s.decode()


@functools.lru_cache(maxsize=None)
def _gapped(name, scale, seed):
    return G.plant_n_runs(seed, G.named_set(name, scale))


KS = [1, 2, 3, 5, 8, 15, 16, 25, 31, 32, 47, 63]


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("both", [True, False])
def test_random_strings_with_n_match_oracle(k, both):
    rng = np.random.default_rng(7000 + k + 100 * both)
    base = [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 6, 0, 2000, b"ACGT")]
    base += [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 3, 40, 600, b"AC")]
    seqs = [_with_ns(rng, s, k) for s in base]
    seqs += ["N" * (k + 2), "", "n", "A" * (k + 3) + "N" + "A" * (k - 1)]
    want = O.junctions(seqs, k, both_strands=both, split_n=True)
    for bits, h, rounds in ((256, 1, 1), (1 << 12, 3, 1), (1 << 18, 8, 1), (1 << 14, 4, 3)):
        got, _ = T().twopaco_build_ex(seqs, k, bits, rounds,
                                      T().Options(hashes=h, both_strands=both, partition_bins=64,
                                                  split_at_n=True))
        _eq(got, want)


def test_n_without_split_is_a_bad_base():
    with pytest.raises(T().TwopacoError) as e:
        T().twopaco_build_ex(["ACGTACGTNACGT"], 3, 1 << 12, 1, T().Options())
    assert e.value.code == -2


def test_split_without_n_changes_nothing():
    seqs = G.named_set("plain_single", 0.05)
    a, sa = T().twopaco_build_ex(seqs, 25, 1 << 20, 1, T().Options(hashes=3))
    b, sb = T().twopaco_build_ex(seqs, 25, 1 << 20, 1, T().Options(hashes=3, split_at_n=True))
    _eq(a, b)
    assert sa["pass1_marks"] == sb["pass1_marks"] and sa["positions"] == sb["positions"]


@pytest.mark.parametrize("k,bits,h", [(25, 1 << 20, 3), (31, 1 << 18, 4), (47, 1 << 20, 8), (15, 1 << 16, 5)])
def test_pass1_candidates_with_n_bit_exact(k, bits, h):
    seqs = _gapped("plain_single", 0.1, 11)
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, k, bits, 1, T().Options(hashes=h, split_at_n=True))
    run.run()
    m = int(off[-1])
    words = run.state(T().STATE_CANDIDATES, (m + 31) // 32)
    ctemp = np.unpackbits(words.view(np.uint8), bitorder="little")[:m]
    marks, _, active, kept = O.pass1_marks((bases, off), k, bits, h, split_n=True)
    assert np.array_equal(ctemp, marks)
    st = run.stats()
    assert st["positions"] == active and st["pass1_marks"] == kept
    _eq(run.result(), O.junctions((bases, off), k, split_n=True))


@pytest.mark.parametrize("name,scale,k", [("plain_single", 0.5, 25), ("bacterial_set", 0.1, 31),
                                          ("batched_set", 0.01, 63), ("bacterial_set", 0.1, 15)])
def test_gapped_genomes_match_oracle(name, scale, k):
    seqs = _gapped(name, scale, 5)
    bases, off = G.concat(seqs)
    want = O.junctions((bases, off), k, split_n=True)
    for rounds in (1, 4):
        run = T().DeviceBuild(bases, off, k, 1 << 24, rounds,
                              T().Options(hashes=4, partition_bins=1024, split_at_n=True,
                                          run_capacity=len(seqs) + 1 + bases.size // 64))
        run.run()
        _eq(run.result(), want)


def test_candidate_list_overflow_with_n_walks_ctemp():
    seqs = _gapped("plain_single", 0.05, 3)
    bases, off = G.concat(seqs)
    got, st = T().twopaco_build_ex(seqs, 25, 1 << 12, 1,
                                   T().Options(hashes=3, candidate_records=300, split_at_n=True))
    _eq(got, O.junctions((bases, off), 25, split_n=True))


def test_run_capacity_overflow_is_reported():
    seqs = ["ACGTN" * 50, "NNACGTACGTNN" * 20]
    bases, off = G.concat([np.frombuffer(s.encode(), np.uint8) for s in seqs])
    run = T().DeviceBuild(bases, off, 3, 1 << 12, 1, T().Options(split_at_n=True, run_capacity=10))
    with pytest.raises(T().TwopacoError) as e:
        run.run()
        run.stats(check=True)
    assert e.value.code == -6
    # the host build counts the boundaries itself, and raises a capacity that is too small
    for cap in (0, 10):
        got, _ = T().twopaco_build_ex(seqs, 3, 1 << 12, 1, T().Options(split_at_n=True, run_capacity=cap))
        _eq(got, O.junctions(seqs, 3, split_n=True))


@pytest.mark.parametrize("k,both", [(3, True), (25, True), (31, False), (63, True)])
def test_edges_with_n_match_oracle(k, both):
    rng = np.random.default_rng(31 + k)
    base = [bytes(s).decode() for s in G.random_strings(900 + k, 8, 0, 1500, b"ACGT")]
    seqs = [_with_ns(rng, s, k) for s in base] + ["N" * 5, "ACGT" * 30 + "N" + "ACGT" * 30]
    seqs += [bytes(s).decode() for s in _gapped("plain_single", 0.02, 9)]
    ctx = T().Context()
    ctx.build(seqs, k, 1 << 20, 1, T().Options(hashes=4, both_strands=both, split_at_n=True))
    off, got = ctx.edges()
    want = O.edges(seqs, k, both_strands=both, split_n=True)
    assert np.array_equal(np.diff(off), want["per_string"])
    for f in ("from_hi", "from_lo", "to_hi", "to_lo", "start", "length", "from_rc", "to_rc"):
        assert np.array_equal(got[f].astype(np.uint64), want[f].astype(np.uint64)), f
    ctx.close()
