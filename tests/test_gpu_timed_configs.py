"""Every configuration the benchmark times, checked at the size it times it.

Each test runs the benchmark's own launch -- the whole build captured once as
a CUDA graph and replayed -- on the full-size input with the parameters the
benchmark uses, and compares the junction positions of every string, element
by element, with the CPU oracle's (the definition of J(S, k), split over the
host's cores by k-mer hash class). Integer work: the comparison is exact.
"""
import os

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


def _cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _eq(got, want):
    assert len(got) == len(want)
    for t, (g, w) in enumerate(zip(got, want)):
        g = np.asarray(g, dtype=np.uint64)
        w = np.asarray(w, dtype=np.uint64)
        if not np.array_equal(g, w):
            raise AssertionError(f"string {t}: {g.size} vs {w.size} junctions; extra "
                                 f"{np.setdiff1d(g, w)[:10]}, missing {np.setdiff1d(w, g)[:10]}")


def _replayed(bases, off, k, bits, hashes, rounds=1, replays=3):
    run = T().DeviceBuild(bases, off, k, bits, rounds, T().Options(hashes=hashes))
    run.capture()
    for _ in range(replays):
        run.run()
    got, st = run.result(), run.stats()
    run.release_plan()
    return got, st


def test_bacterial_set_as_benchmarked():
    """7 genomes of 4.6-5.6 Mbp (35.4 Mbp), k = 25, 2^28 bits, 4 hashes, 1 round, graph replay."""
    bases, off = G.concat(G.named_set("bacterial_set"))
    got, st = _replayed(bases, off, 25, 1 << 28, 4)
    want = O.junctions((bases, off), 25, threads=_cores())
    _eq(got, want)
    assert st["pass2_marks"] == sum(w.size for w in want)


def test_batched_set_full_size_as_benchmarked():
    """The 62-genome set at full size (310 Mbp), k = 25, with the filter the benchmark's
    tuner settles on for it (2^30 bits, 4 hashes), graph replay."""
    bases, off = G.concat(G.named_set("batched_set"))
    assert int(off[-1]) > 300_000_000
    got, st = _replayed(bases, off, 25, 1 << 30, 4, replays=2)
    want = O.junctions((bases, off), 25, threads=_cores())
    _eq(got, want)
    assert st["pass2_marks"] == sum(w.size for w in want)
    assert st["positions"] == sum(int(off[t + 1] - off[t]) - 24 for t in range(len(off) - 1))
