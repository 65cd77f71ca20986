"""k > 63 on the GPU (four-word k-mers, reference slots) against the oracle.

Bit-exact junction positions per string, the pass-1 candidate bitmap, and
the compacted-graph edges (whose from/to words carry the last 64 bases of
each normalized k-mer), for k from 64 to 127 -- k = 100 is the paper's
long-k setting (Tables 2-4).
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


@functools.lru_cache(maxsize=None)
def _named(name, scale):
    return G.named_set(name, scale)


def _revcomp(s):
    return s.translate(str.maketrans("ACGT", "TGCA"))[::-1]


@pytest.mark.parametrize("k", [64, 65, 70, 96, 97, 100, 120, 127])
@pytest.mark.parametrize("both", [True, False])
def test_random_strings_match_oracle(k, both):
    rng = np.random.default_rng(8100 + k + 1000 * both)
    seqs = [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 6, 0, 3000, b"ACGT")]
    seqs += [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 3, k, 5 * k, b"AC")]
    seqs.append(_revcomp(seqs[0]))
    seqs.append(seqs[1][100:900] + seqs[2][:400])
    seqs += ["A" * (k + 5), "ACGT" * (k // 2), "C" * (k - 1)]
    want = O.junctions(seqs, k, both_strands=both)
    for bits, h, rounds in ((256, 1, 1), (1 << 12, 3, 1), (1 << 18, 8, 1), (1 << 14, 4, 3)):
        got, _ = T().twopaco_build_ex(seqs, k, bits, rounds,
                                      T().Options(hashes=h, both_strands=both, partition_bins=64))
        _eq(got, want)


@pytest.mark.parametrize("k,bits,h", [(100, 1 << 20, 4), (127, 1 << 18, 7), (64, 1 << 16, 2)])
def test_pass1_candidates_bit_exact(k, bits, h):
    seqs = _named("plain_single", 0.1)
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, k, bits, 1, T().Options(hashes=h))
    run.run()
    m = int(off[-1])
    words = run.state(T().STATE_CANDIDATES, (m + 31) // 32)
    ctemp = np.unpackbits(words.view(np.uint8), bitorder="little")[:m]
    marks, _, active, kept = O.pass1_marks((bases, off), k, bits, h)
    assert np.array_equal(ctemp, marks)
    st = run.stats()
    assert st["positions"] == active and st["pass1_marks"] == kept
    _eq(run.result(), O.junctions((bases, off), k))


@pytest.mark.parametrize("name,scale,rounds", [("batched_set", 0.02, 1), ("bacterial_set", 0.05, 4),
                                               ("plain_single", 0.5, 1)])
def test_genome_sets_k100(name, scale, rounds):
    seqs = _named(name, scale)
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, 100, 1 << 24, rounds, T().Options(hashes=4, partition_bins=1024))
    run.run()
    _eq(run.result(), O.junctions((bases, off), 100))


def test_small_table_and_list_overflow_k100():
    seqs = _named("plain_single", 0.05)
    bases, off = G.concat(seqs)
    want = O.junctions((bases, off), 100)
    got, st = T().twopaco_build_ex(seqs, 100, 1 << 16, 1, T().Options(hashes=3, table_slots=1024))
    _eq(got, want)
    assert st["table_slots"] > 1024
    got, _ = T().twopaco_build_ex(seqs, 100, 1 << 12, 1, T().Options(hashes=3, candidate_records=300))
    _eq(got, want)


def test_split_n_k100():
    seqs = G.plant_n_runs(21, _named("plain_single", 0.1))
    bases, off = G.concat(seqs)
    got, _ = T().twopaco_build_ex(seqs, 100, 1 << 22, 2, T().Options(hashes=4, partition_bins=256,
                                                                      split_at_n=True))
    _eq(got, O.junctions((bases, off), 100, split_n=True))


@pytest.mark.parametrize("k,both", [(64, True), (100, True), (127, False)])
def test_edges_long_k_match_oracle(k, both):
    seqs = _named("plain_single", 0.02)
    ctx = T().Context()
    ctx.build(seqs, k, 1 << 20, 1, T().Options(hashes=4, both_strands=both))
    off, got = ctx.edges()
    want = O.edges(G.concat(seqs), k, both_strands=both)
    assert np.array_equal(np.diff(off), want["per_string"])
    for f in ("from_hi", "from_lo", "to_hi", "to_lo", "start", "length", "from_rc", "to_rc"):
        assert np.array_equal(got[f].astype(np.uint64), want[f].astype(np.uint64)), f
    ctx.close()


def test_captured_run_k100():
    seqs = _named("plain_single", 0.05)
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, 100, 1 << 20, 2, T().Options(hashes=4, partition_bins=256))
    run.capture()
    for _ in range(2):
        run.run()
    _eq(run.result(), O.junctions((bases, off), 100))
    run.release_plan()
