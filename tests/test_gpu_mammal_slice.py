"""The mammal-scale configuration at slice scale (8 tree-related genomes, 45%
repeats, 1-8% divergence; k = 25): bit-exact against the oracle for rounds in
{1, 4, 16} and two filter sizes -- the slice's analogues of 2^34 and 2^36 bits
(about 1 and 4 bits per base) -- through the host API, which copies the
strings from host memory.
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


@functools.lru_cache(maxsize=None)
def _slice():
    seqs = G.mammal_slice(genome_len=500_000)
    return seqs, O.junctions(G.concat(seqs), 25)


@pytest.mark.parametrize("rounds", [1, 4, 16])
@pytest.mark.parametrize("bits", [1 << 22, 1 << 24])
def test_mammal_slice_matches_oracle(rounds, bits):
    from paper_1602_05856_gb300 import twopaco as T
    seqs, want = _slice()
    got, st = T.twopaco_build_ex(seqs, 25, bits, rounds, T.Options(hashes=4, partition_bins=4096))
    assert len(got) == len(want)
    for g, w in zip(got, want):
        assert np.array_equal(np.asarray(g, np.uint64), np.asarray(w, np.uint64))
    assert st["pass2_marks"] == sum(w.size for w in want)


def test_mammal_slice_device_resident_rounds_agree():
    from paper_1602_05856_gb300 import twopaco as T
    seqs, want = _slice()
    bases, off = G.concat(seqs)
    results = []
    for rounds in (1, 16):
        run = T.DeviceBuild(bases, off, 25, 1 << 24, rounds, T.Options(hashes=4, partition_bins=4096))
        run.run()
        results.append(run.result())
    for a, b, w in zip(results[0], results[1], want):
        assert np.array_equal(a, b) and np.array_equal(a, np.asarray(w, np.uint64))
