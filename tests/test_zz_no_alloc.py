"""The entry point that allocates nothing, against the workspace entry point.

twopaco_run_device_noalloc serves callers that may not allocate device
memory (their host framework's pool owns it all, or cudaMalloc's implicit
synchronisation is not affordable): its workspace is a fixed static device
buffer. This test calls it twice in a row through the C ABI and checks both
results, element by element, against twopaco_run_device with a workspace
allocated here and against the CPU oracle's junctions, and that an input too
large for the buffer is rejected. Junction positions are integers: the
comparison is exact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_05856_gb300 import build, twopaco
    build.build()
    twopaco.load()
    return twopaco


def _device_input(seqs):
    import torch
    from paper_1602_05856_gb300 import genomes
    bases, off = genomes.concat(seqs)
    d_bases = torch.from_numpy(bases).cuda()
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    return bases, off, d_bases, d_off


def _outputs(n_seqs, capacity):
    import torch
    return (torch.zeros(n_seqs + 1, dtype=torch.int64, device="cuda"),
            torch.full((capacity,), -1, dtype=torch.int64, device="cuda"))


def _split(out_off, out_pos):
    off = out_off.cpu().numpy().view(np.uint64)
    pos = out_pos[: int(off[-1])].cpu().numpy().view(np.uint64)
    return off, pos


def test_noalloc_matches_workspace_run_twice(lib):
    import torch
    from paper_1602_05856_gb300 import genomes
    T = lib
    k, bits, rounds = 25, 1 << 20, 1
    opts = T.Options(hashes=4, table_slots=1 << 20, candidate_records=1 << 18)
    seqs = genomes.named_set("plain_single", scale=0.05)  # 4 related genomes, ~50 kbp each
    bases, off, d_bases, d_off = _device_input(seqs)
    m, n = bases.size, len(seqs)

    # reference: the workspace entry point, workspace allocated by the caller
    ws_bytes = T.twopaco_workspace_size(m, n, k, bits, rounds, opts)
    assert ws_bytes <= T.NOALLOC_SCRATCH_BYTES
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device="cuda")
    ws_ptr = (ws.data_ptr() + 255) // 256 * 256
    ref_off, ref_pos = _outputs(n, m)
    T.twopaco_run_device(d_bases.data_ptr(), d_off.data_ptr(), n, m, k, bits, rounds, opts, ws_ptr,
                         ws_bytes, ref_off.data_ptr(), ref_pos.data_ptr(), m)
    ref_stats = T.twopaco_read_stats(ws_ptr)
    want_off, want_pos = _split(ref_off, ref_pos)
    assert want_pos.size > 0
    import oracle as O
    by_definition = O.junctions((bases, off), k)
    assert np.array_equal(np.diff(want_off.astype(np.int64)), [w.size for w in by_definition])
    assert np.array_equal(want_pos, np.concatenate(by_definition))

    # the entry point that allocates nothing, twice in a row on the same buffer
    for _ in range(2):
        out_off, out_pos = _outputs(n, m)
        st = T.twopaco_run_device_noalloc(d_bases.data_ptr(), d_off.data_ptr(), n, m, k, bits, rounds,
                                          opts, out_off.data_ptr(), out_pos.data_ptr(), m)
        got_off, got_pos = _split(out_off, out_pos)
        assert np.array_equal(got_off, want_off)
        assert np.array_equal(got_pos, want_pos)
        for key in ("positions", "pass1_marks", "pass2_marks"):
            assert st[key] == ref_stats[key]


def test_noalloc_rejects_inputs_beyond_its_buffer(lib):
    import torch
    T = lib
    m = 10_000_000  # a 2^28-bit filter alone is 32 MiB
    big = T.twopaco_workspace_size(m, 1, 25, 1 << 28, 1)
    assert big > T.NOALLOC_SCRATCH_BYTES
    d_bases = torch.zeros(16, dtype=torch.uint8, device="cuda")
    d_off = torch.tensor([0, m], dtype=torch.int64, device="cuda")
    out_off, out_pos = _outputs(1, 16)
    with pytest.raises(T.TwopacoError) as e:
        T.twopaco_run_device_noalloc(d_bases.data_ptr(), d_off.data_ptr(), 1, m, 25, 1 << 28, 1, None,
                                     out_off.data_ptr(), out_pos.data_ptr(), 16)
    assert e.value.code == T.ESCRATCH
