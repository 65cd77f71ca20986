"""The run that streams its input from host memory, and the mammal-scale recipe drawn on the GPU.

twopaco_run_streamed copies the input in chunks through a two-half staging
buffer while packing the chunk before; its junctions must be the oracle's,
element by element, for any chunk size (ragged last chunk, chunks smaller
than a string, N masks across chunk boundaries, rounds, long k).

The mammal-scale configuration is drawn on the GPU (genomes_gpu); at slice
size (8 leaves of tens of Mbp) the GPU's junctions must be the oracle's for
rounds 1, 4 and 16 and two filter sizes, and the streamed run must agree.
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
        assert np.array_equal(np.asarray(g, np.uint64), np.asarray(w, np.uint64)), t


def _streamed(bases, off, k, bits, rounds, opts, half_bytes):
    import torch
    host = torch.empty(bases.size, dtype=torch.uint8, pin_memory=True)
    host.numpy()[:] = bases
    run = T().DeviceBuild(bases, off, k, bits, rounds, opts, resident=False)
    staging = torch.empty(2 * half_bytes, dtype=torch.uint8, device="cuda")
    run.run_streamed(host, staging)
    return run


@pytest.mark.parametrize("half", [64 << 10, (64 << 10) + 256, 1 << 20, 64 << 20])
def test_streamed_run_matches_oracle(half):
    bases, off = G.concat(G.named_set("plain_single", 0.3))
    run = _streamed(bases, off, 25, 1 << 22, 1, T().Options(hashes=4), half)
    _eq(run.result(), O.junctions((bases, off), 25, threads=_cores()))
    st = run.stats()
    assert st["positions"] == sum(int(off[t + 1] - off[t]) - 24 for t in range(len(off) - 1))


@pytest.mark.parametrize("k,rounds,split", [(31, 4, False), (21, 3, True), (100, 2, False), (25, 1, True)])
def test_streamed_rounds_split_and_long_k(k, rounds, split):
    seqs = G.named_set("plain_single", 0.1)
    if split:
        seqs = G.plant_n_runs(21, seqs)
    bases, off = G.concat(seqs)
    opts = T().Options(hashes=4, partition_bins=1024, split_at_n=split)
    run = _streamed(bases, off, k, 1 << 20, rounds, opts, 64 << 10)
    _eq(run.result(), O.junctions((bases, off), k, split_n=split, threads=_cores()))


def test_streamed_bad_base_index_across_chunks():
    bases, off = G.concat(G.named_set("plain_single", 0.05))
    bases = bases.copy()
    bad = 3 * (64 << 10) + 77  # in the fourth chunk
    bases[bad] = ord("X")
    run = _streamed(bases, off, 25, 1 << 20, 1, T().Options(), 64 << 10)
    st = run.stats(check=False)
    assert st["rc"] == T().EBADBASE and st["bad_base_index"] == bad


def test_streamed_staging_too_small_is_refused():
    import torch
    bases, off = G.concat(G.named_set("plain_single", 0.01))
    run = T().DeviceBuild(bases, off, 25, 1 << 20, 1, resident=False)
    staging = torch.empty(64 << 10, dtype=torch.uint8, device="cuda")  # two halves of 32 KiB
    with pytest.raises(T().TwopacoError) as e:
        run.run_streamed(bases, staging)
    assert e.value.code == T().EINVAL
    with pytest.raises(ValueError):
        run.run()  # the bases are not resident


def test_mammal_slice_drawn_on_gpu_matches_oracle():
    """8 leaves of 25 Mbp from the GPU-drawn mammal-scale recipe (45% repeats at 10-15%
    divergence, 1-8% between leaves): rounds 1, 4, 16 and 1 or 4 filter bits per base
    against the oracle, and the streamed run against the resident one."""
    import torch
    from paper_1602_05856_gb300 import genomes_gpu as GG
    leaves = GG.mammal_set(genome_len=25_000_000)
    d_bases, off = GG.concat_device(leaves)
    del leaves
    bases = d_bases.cpu().numpy()
    m = int(off[-1])
    want = O.junctions((bases, off), 25, threads=_cores())
    n_j = sum(w.size for w in want)
    assert 0.03 < n_j / m < 0.4  # a branching graph, as the recipe intends
    for rounds, bits in ((1, 1 << 28), (4, 1 << 28), (16, 1 << 26), (4, 1 << 26)):
        opts = T().Options(hashes=4, table_slots=m // 2, candidate_records=m // 2)
        run = T().DeviceBuild(d_bases, off, 25, bits, rounds, opts, capacity=m // 2)
        run.run()
        _eq(run.result(), want)
        del run
    host = torch.empty(m, dtype=torch.uint8, pin_memory=True)
    host.numpy()[:] = bases
    run = T().DeviceBuild(d_bases, off, 25, 1 << 28, 4,
                          T().Options(hashes=4, table_slots=m // 2, candidate_records=m // 2),
                          capacity=m // 2, resident=False)
    run.run_streamed(host, torch.empty(2 << 26, dtype=torch.uint8, device="cuda"))
    _eq(run.result(), want)
