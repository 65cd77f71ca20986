"""Round ranges and checkpoints (per-round resume) on the GPU.

A run split into round ranges, or stopped after any round, saved, restored
into a fresh workspace and finished, gives the same junctions (bit-exact vs
the oracle) and the same counters as the run in one go; a checkpoint of
another input or parameter set is refused.
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
    for g, w in zip(got, want):
        assert np.array_equal(np.asarray(g, np.uint64), np.asarray(w, np.uint64))


@functools.lru_cache(maxsize=None)
def _input(scale=0.1, split=False):
    seqs = G.named_set("plain_single", scale)
    if split:
        seqs = G.plant_n_runs(3, seqs)
    return G.concat(seqs)


KEYS = ("positions", "pass1_marks", "pass2_marks", "table_slots")
# The class cut comes from a Bloom pre-pass whose counters are order-dependent
# (two first occurrences of a k-mer processed at once may both count), so two
# separate runs with rounds > 1 may split the k-mers differently: their
# junctions agree, but pass-1 marks and table sizes need not. These do not
# depend on the cut:
CUT_FREE = ("positions", "pass2_marks")


def _build(k, rounds, **opt):
    bases, off = _input(split=opt.get("split_at_n", False))
    return T().DeviceBuild(bases, off, k, 1 << 20, rounds,
                           T().Options(hashes=4, partition_bins=256, **opt))


def test_round_ranges_equal_one_run():
    full = _build(25, 5)
    full.run()
    want_st = full.stats()
    part = _build(25, 5)
    part.run_rounds(0, 2)
    part.run_rounds(2, 3)
    part.run_rounds(3, 5)
    _eq(part.result(), full.result())
    st = part.stats()
    assert {x: st[x] for x in CUT_FREE} == {x: want_st[x] for x in CUT_FREE}
    _eq(part.result(), O.junctions(_input(), 25))


@pytest.mark.parametrize("stop", [1, 2, 4, 5])
def test_checkpoint_restore_in_a_fresh_workspace(stop, tmp_path):
    a = _build(31, 5)
    a.run_rounds(0, stop)
    blob = a.checkpoint(stop)
    path = tmp_path / "run.ckpt"
    path.write_bytes(blob)
    if stop < 5:
        a.run_rounds(stop, 5)  # the run that was not interrupted, with the same class cut
    want, want_st = a.result(), a.stats()
    _eq(want, O.junctions(_input(), 31))
    b = _build(31, 5)  # another workspace, as after a restart
    nxt = b.restore(path.read_bytes())
    assert nxt == stop
    b.run_rounds(nxt, 5)
    _eq(b.result(), want)
    st = b.stats()
    assert {x: st[x] for x in KEYS} == {x: want_st[x] for x in KEYS}


def test_checkpoint_split_n_long_k():
    full = _build(100, 3, split_at_n=True)
    full.run()
    a = _build(100, 3, split_at_n=True)
    a.run_rounds(0, 2)
    blob = a.checkpoint(2)
    b = _build(100, 3, split_at_n=True)
    b.run_rounds(b.restore(blob), 3)
    _eq(b.result(), full.result())
    _eq(b.result(), O.junctions(_input(split=True), 100, split_n=True))


def test_foreign_checkpoints_are_refused():
    a = _build(25, 4)
    a.run_rounds(0, 2)
    blob = a.checkpoint(2)
    with pytest.raises(T().TwopacoError) as e:  # other k
        _build(27, 4).restore(blob)
    assert e.value.code == T().EINVAL
    with pytest.raises(T().TwopacoError) as e:  # other round count
        _build(25, 5).restore(blob)
    assert e.value.code == T().EINVAL
    bases, off = _input()
    other = bases.copy()
    other[1000] = ord("A") if other[1000] != ord("A") else ord("C")  # one base differs
    c = T().DeviceBuild(other, off, 25, 1 << 20, 4, T().Options(hashes=4, partition_bins=256))
    with pytest.raises(T().TwopacoError) as e:
        c.restore(blob)
    assert e.value.code == T().EINVAL
    bad = bytearray(blob)
    bad[0] ^= 1
    with pytest.raises(T().TwopacoError):
        _build(25, 4).restore(bytes(bad))
    for at in (len(blob) - 1, len(blob) // 2):  # a payload bit changed after saving
        bad = bytearray(blob)
        bad[at] ^= 4
        with pytest.raises(T().TwopacoError) as e:
            _build(25, 4).restore(bytes(bad))
        assert e.value.code == T().EINVAL
    _build(25, 4).restore(blob)  # the undamaged checkpoint still loads
    with pytest.raises(T().TwopacoError):
        _build(25, 4).restore(blob[: len(blob) // 2])
    # the genuine one still works
    d = _build(25, 4)
    d.run_rounds(d.restore(blob), 4)
    _eq(d.result(), O.junctions(_input(), 25))


# Byte offsets of head fields in a checkpoint (the head is 128 bytes: magic,
# version, nine int32 parameters, then 64-bit fields).
NEXT_ROUND_AT, POSITIONS_AT, PASS2_AT = 32, 88, 104


def test_changed_head_fields_are_refused():
    """The checksum covers the head: a resume point or counter edited after saving is
    refused (a next_round moved from 2 to 3 would otherwise skip round 2 silently)."""
    import struct
    a = _build(25, 4)
    a.run_rounds(0, 2)
    blob = a.checkpoint(2)
    assert struct.unpack_from("<i", blob, NEXT_ROUND_AT)[0] == 2
    for at, fmt, value in ((NEXT_ROUND_AT, "<i", 3), (POSITIONS_AT, "<Q", 12345),
                           (PASS2_AT, "<Q", 1)):
        bad = bytearray(blob)
        struct.pack_into(fmt, bad, at, value)
        with pytest.raises(T().TwopacoError) as e:
            _build(25, 4).restore(bytes(bad))
        assert e.value.code == T().EINVAL
    b = _build(25, 4)
    b.run_rounds(b.restore(blob), 4)
    _eq(b.result(), O.junctions(_input(), 25))


def test_checkpoint_of_moved_boundaries_is_refused():
    """Same bases, same number of strings, other string boundaries: other sentinels and
    other edges, so the digest (which covers the offsets) differs."""
    bases, off = _input()
    a = T().DeviceBuild(bases, off, 25, 1 << 20, 3, T().Options(hashes=4, partition_bins=256))
    a.run_rounds(0, 1)
    blob = a.checkpoint(1)
    moved = off.copy()
    moved[1] += 7
    b = T().DeviceBuild(bases, moved, 25, 1 << 20, 3, T().Options(hashes=4, partition_bins=256))
    with pytest.raises(T().TwopacoError) as e:
        b.restore(blob)
    assert e.value.code == T().EINVAL
    c = T().DeviceBuild(bases, off, 25, 1 << 20, 3, T().Options(hashes=4, partition_bins=256))
    c.run_rounds(c.restore(blob), 3)
    _eq(c.result(), O.junctions((bases, off), 25))


def test_checkpoint_of_g_and_n_swapped_is_refused():
    """With split_at_n an N packs to G's code; the digest covers the N mask, so an input
    with one G changed to N (or back) does not pass for the one checkpointed."""
    bases, off = _input(split=True)
    opts = T().Options(hashes=4, partition_bins=256, split_at_n=True)
    a = T().DeviceBuild(bases, off, 25, 1 << 20, 3, opts)
    a.run_rounds(0, 2)
    blob = a.checkpoint(2)
    g_at = int(np.flatnonzero(bases == ord("G"))[100])
    n_at = int(np.flatnonzero((bases == ord("N")) | (bases == ord("n")))[0])
    for at, byte in ((g_at, ord("N")), (n_at, ord("G"))):
        other = bases.copy()
        other[at] = byte
        b = T().DeviceBuild(other, off, 25, 1 << 20, 3, opts)
        with pytest.raises(T().TwopacoError) as e:
            b.restore(blob)
        assert e.value.code == T().EINVAL
    c = T().DeviceBuild(bases, off, 25, 1 << 20, 3, opts)
    c.run_rounds(c.restore(blob), 3)
    _eq(c.result(), O.junctions((bases, off), 25, split_n=True))


def test_finished_run_output_from_its_last_checkpoint():
    a = _build(25, 2)
    a.run()
    blob = a.checkpoint(2)
    b = _build(25, 2)
    assert b.restore(blob) == 2
    b.run_rounds(2, 2)  # only writes the output
    _eq(b.result(), a.result())


def test_output_too_small_then_written_again():
    """A run whose output does not fit reports its exact junction count; after a larger
    buffer is given, twopaco_run_rounds(rounds, rounds) writes the output again."""
    import torch
    bases, off = _input()
    run = _build(25, 3)
    small = torch.empty(10, dtype=torch.int64, device="cuda")
    T().twopaco_run_device(run.bases.data_ptr(), run.offsets.data_ptr(), run.n_seqs, run.total_bases,
                           25, 1 << 20, 3, T().Options(hashes=4, partition_bins=256), run.ws_ptr,
                           run.ws_bytes, run.out_offsets.data_ptr(), small.data_ptr(), 10)
    st = run.stats(check=False)
    assert st["rc"] == T().EOVERFLOW and st["overflow"]
    total = int(run.out_offsets.cpu().numpy().view(np.uint64)[-1])
    want = O.junctions(_input(), 25)
    assert total == sum(w.size for w in want) > 10
    run.run_rounds(3, 3)  # into the build's own buffer (room for every position)
    _eq(run.result(), want)
    assert run.stats()["rc"] == 0
