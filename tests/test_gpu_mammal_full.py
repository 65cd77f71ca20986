"""The mammal-scale configuration at full size (8 genomes of 3 Gbp, 24 Gbp), by invariants.

The CPU oracle cannot hold this input's k-mers, so at full size the output is
checked by what must hold at any size (the slice is checked against the
oracle in test_gpu_streamed.py):

* the junctions do not depend on the rounds or on the filter: rounds 4 and 16
  with 2^36 bits, and rounds 4 with 2^34 bits, give identical output;
* they equal the output of a run whose filter is saturated (256 bits: every
  position survives the first pass), in which the exact second pass alone
  decides every position -- Algorithm 1 with an exact edge set;
* the first and last k-mer of every genome are junctions (sentinels), and the
  streamed run from host memory gives the resident run's output.

Outputs are compared through a digest computed on the device (the sum of a
mix of every junction's global position), plus the per-genome counts.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GENOME_LEN = 3_000_000_000
K = 25


@pytest.fixture(scope="module")
def mammal():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if total < 250 << 30:
        pytest.skip("needs a device of 250 GB or more")
    from paper_1602_05856_gb300 import build, genomes_gpu as GG
    build.build()
    leaves = GG.mammal_set(genome_len=GENOME_LEN)
    d_bases, off = GG.concat_device(leaves)
    del leaves
    torch.cuda.empty_cache()
    yield d_bases, off
    del d_bases
    torch.cuda.empty_cache()


def _digest(run):
    """(junctions per genome, order-free digest of the global junction positions), computed
    per genome in slices so that no temporary holds the whole output."""
    st = run.stats()
    off = run.out_offsets.cpu().numpy().view(np.uint64)
    starts = run.offsets.cpu().numpy()
    per = np.diff(off).astype(np.int64)
    h = 0
    step = 1 << 27
    for t in range(len(per)):
        a, b = int(off[t]), int(off[t + 1])
        for c in range(a, b, step):
            g = run.out_positions[c:min(b, c + step)] + int(starts[t])
            h += int(((g * 0x5851F42D4C957F2D) ^ (g >> 29)).sum().item())
    return per.tolist(), h % (1 << 64), st, None


def _run(d_bases, off, bits, rounds, table_slots, records):
    from paper_1602_05856_gb300 import twopaco as T
    m = int(off[-1])
    opts = T.Options(hashes=4, table_slots=table_slots, candidate_records=records)
    run = T.DeviceBuild(d_bases, off, K, bits, rounds, opts, capacity=m // 3)
    run.run()
    return run


def test_mammal_full_size_invariants(mammal):
    import torch
    from paper_1602_05856_gb300 import twopaco as T
    d_bases, off = mammal
    m = int(off[-1])
    assert m > 23_000_000_000
    digests = {}
    for bits, rounds, slots, recs in ((1 << 36, 4, 1 << 31, m // 8), (1 << 36, 16, 1 << 30, m // 32),
                                      (1 << 34, 4, 1 << 31, m // 8)):
        run = _run(d_bases, off, bits, rounds, slots, recs)
        per, dig, st, pos = _digest(run)
        digests[(bits, rounds)] = (per, dig)
        o = run.out_offsets.cpu().numpy().view(np.uint64)
        for t in range(len(off) - 1):  # sentinels: first and last k-mer of every genome
            assert int(run.out_positions[int(o[t])].item()) == 0
            assert int(run.out_positions[int(o[t + 1]) - 1].item()) == int(off[t + 1] - off[t]) - K
        del run, pos
        torch.cuda.empty_cache()
    vals = list(digests.values())
    assert all(v == vals[0] for v in vals), digests
    # every position survives a 256-bit filter: pass 2 alone decides, exactly
    run = _run(d_bases, off, 256, 16, 1 << 31, m // 16 + (1 << 20))
    per, dig, st, _ = _digest(run)
    assert st["pass1_marks"] == st["positions"]
    assert (per, dig) == vals[0]
    del run
    torch.cuda.empty_cache()
    # the streamed run from host memory
    host = torch.empty(m, dtype=torch.uint8, pin_memory=True)
    host.copy_(d_bases)
    opts = T.Options(hashes=4, table_slots=1 << 31, candidate_records=m // 8)
    run = T.DeviceBuild(d_bases, off, K, 1 << 36, 4, opts, capacity=m // 3, resident=False)
    run.run_streamed(host, torch.empty(1 << 29, dtype=torch.uint8, device="cuda"))
    per, dig, _, _ = _digest(run)
    assert (per, dig) == vals[0]
