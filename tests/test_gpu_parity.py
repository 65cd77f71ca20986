"""GPU path vs the CPU oracle, through the C ABI. Integer work: bit-exact.

Every comparison is element by element: the junction positions of every
string, and (where stated) the pass-1 candidate bitmap C_temp against the
oracle's restatement of the same filter.
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
        if not np.array_equal(g, w):
            extra = np.setdiff1d(g, w)[:10]
            miss = np.setdiff1d(w, g)[:10]
            raise AssertionError(f"string {t}: {g.size} vs {w.size} junctions; "
                                 f"extra {extra}, missing {miss}")


def _bits_to_marks(words: np.ndarray, m: int) -> np.ndarray:
    b = np.unpackbits(words.view(np.uint8), bitorder="little")
    return b[:m]


@functools.lru_cache(maxsize=None)
def _named(name, scale):
    return G.named_set(name, scale)


@functools.lru_cache(maxsize=None)
def _oracle_named(name, scale, k):
    seqs = _named(name, scale)
    return O.junctions(G.concat(seqs), k)


# --- worked example ----------------------------------------------------------

@pytest.mark.parametrize("both,k,want", [
    (False, 2, [[0, 4, 7], [0, 4, 7]]),
    (True, 2, [[0, 2, 3, 4, 6, 7], [0, 2, 3, 4, 7]]),
    (True, 3, [[0, 3, 4, 5, 6], [0, 3, 6]]),
])
def test_fig1_worked_example(both, k, want):
    for bits, h in ((256, 1), (1 << 16, 4)):
        got, st = T().twopaco_build_ex(["TGGCACGTC", "TGGCACTTC"], k, bits, 1,
                                       T().Options(hashes=h, both_strands=both))
        _eq(got, want)
        assert st["pass2_marks"] == sum(len(w) for w in want)


# --- random small inputs, every k path -------------------------------------------

KS = [1, 2, 3, 4, 5, 7, 8, 12, 15, 16, 17, 24, 25, 31, 32, 33, 40, 47, 48, 62, 63]


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("both", [True, False])
def test_random_inputs_match_oracle(k, both):
    rng = np.random.default_rng(1000 + k + 100 * both)
    seqs = [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 6, 0, 3000,
                                                        b"ACGT")]
    seqs += [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 3, 50, 700,
                                                         b"AC")]
    seqs.append(brute.revcomp(seqs[0]))
    seqs.append(seqs[1][100:900] + seqs[2][:400])
    seqs.append("A" * (k + 5))
    want = O.junctions(seqs, k, both_strands=both)
    for bits, h, rounds in ((256, 1, 1), (1 << 12, 3, 1), (1 << 18, 8, 1), (1 << 14, 4, 3)):
        got, _ = T().twopaco_build_ex(seqs, k, bits, rounds,
                                      T().Options(hashes=h, both_strands=both, partition_bins=64))
        _eq(got, want)


def test_small_strings_match_brute_force():
    for seed in range(20):
        k = 1 + seed % 9
        seqs = [bytes(s).decode() for s in G.random_strings(seed, 4, 0, 40, b"ACG")]
        got, _ = T().twopaco_build_ex(seqs, k, 1 << 10, 1, T().Options(hashes=2))
        _eq(got, brute.junction_positions(seqs, k, True))


# --- pass 1 against the oracle's model of the same filter ------------------------

@pytest.mark.parametrize("k,bits,h,both", [(25, 1 << 20, 3, True), (31, 1 << 18, 4, True),
                                           (9, 1 << 14, 2, False), (47, 1 << 20, 8, True),
                                           (63, 1 << 16, 5, True)])
def test_pass1_candidates_bit_exact(k, bits, h, both):
    seqs = _named("plain_single", 0.1)
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, k, bits, 1, T().Options(hashes=h, both_strands=both))
    run.run()
    got = run.result()
    st = run.stats()
    m = int(off[-1])
    ctemp = _bits_to_marks(run.state(T().STATE_CANDIDATES, (m + 31) // 32), m)
    marks, _, active, kept = O.pass1_marks((bases, off), k, bits, h, both_strands=both)
    assert np.array_equal(ctemp, marks)
    assert st["pass1_marks"] == kept and st["positions"] == active
    _eq(got, O.junctions((bases, off), k, both_strands=both))


# --- the named workloads ------------------------------------------------------------

def test_plain_single_full_size():
    """4 related 1 Mbp genomes, k=25, 2^24-bit filter, 3 hashes, 1 round."""
    seqs = _named("plain_single", 1.0)
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, 25, 1 << 24, 1, T().Options(hashes=3))
    run.run()
    _eq(run.result(), _oracle_named("plain_single", 1.0, 25))
    m = int(off[-1])
    ctemp = _bits_to_marks(run.state(T().STATE_CANDIDATES, (m + 31) // 32), m)
    marks, _, _, kept = O.pass1_marks((bases, off), 25, 1 << 24, 3)
    assert np.array_equal(ctemp, marks) and run.stats()["pass1_marks"] == kept


@pytest.mark.parametrize("k", [25, 31])
def test_bacterial_set_full_size(k):
    """7 genomes of 4.6-5.6 Mbp, 2^28-bit filter, 4 hashes: the benchmarked launch."""
    seqs = _named("bacterial_set", 1.0)
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, k, 1 << 28, 1, T().Options(hashes=4))
    run.run()
    run.run()  # a second run on the same workspace must not see the first
    _eq(run.result(), _oracle_named("bacterial_set", 1.0, k))


@pytest.mark.parametrize("k", [15, 25, 31, 63])
def test_batched_set_scaled(k):
    """62 uneven genomes (scaled to ~250 kbp each) for every k of the batched workload."""
    seqs = _named("batched_set", 0.05)
    got, st = T().twopaco_build_ex(seqs, k, 1 << 24, 1, T().Options(hashes=4))
    _eq(got, _oracle_named("batched_set", 0.05, k))


# --- invariances -------------------------------------------------------------------

def test_rounds_filter_and_hash_invariance():
    seqs = _named("plain_single", 0.25)
    bases, off = G.concat(seqs)
    want = O.junctions((bases, off), 25)
    for bits, h, rounds in ((1 << 22, 4, 1), (1 << 22, 4, 2), (1 << 20, 3, 4), (1 << 16, 2, 16),
                            (256, 1, 1), (1 << 26, 8, 5), (1 << 22, 6, 7)):
        run = T().DeviceBuild(bases, off, 25, bits, rounds,
                              T().Options(hashes=h, partition_bins=1024))
        run.run()
        _eq(run.result(), want)
        st = run.stats()
        assert st["pass2_marks"] == sum(w.size for w in want)
        if rounds > 1:
            bins = run.state(T().STATE_BINS, 1024)
            cuts = run.state(T().STATE_CUTS, rounds + 1)
            assert list(cuts) == [int(c) for c in O.partition_cuts(bins, rounds)]
            # the counters count distinct k-mers, less those the pre-pass filter
            # already showed as present
            assert int(bins.sum()) <= O.junction_flags((bases, off), 25)[2]


# --- edge cases ---------------------------------------------------------------------

def test_empty_and_short_inputs():
    got, st = T().twopaco_build_ex([], 25, 1 << 16, 1)
    assert got == [] and st["pass2_marks"] == 0
    got, st = T().twopaco_build_ex(["", "ACGT", "A" * 24], 25, 1 << 16, 1)
    assert [g.size for g in got] == [0, 0, 0] and st["positions"] == 0
    got, _ = T().twopaco_build_ex(["ACGTACGTAC", "CCCCCCCCCC", "A"], 10, 1 << 16, 1)
    _eq(got, [[0], [0], []])


def test_many_tiny_strings():
    rng = np.random.default_rng(5)
    seqs = [bytes(s).decode() for s in G.random_strings(77, 3000, 0, 60, b"ACGT")]
    for i in range(0, 3000, 7):  # shared pieces, so junctions appear inside strings
        seqs[i] = seqs[i][:30] + seqs[(i * 13) % 3000][:40]
    k = int(rng.integers(11, 16))
    got, _ = T().twopaco_build_ex(seqs, k, 1 << 16, 1, T().Options(hashes=3))
    _eq(got, O.junctions(seqs, k))


def test_lowercase_input():
    seqs = [bytes(s).decode() for s in G.random_strings(8, 3, 500, 900, b"ACGT")]
    low = [s.lower() if i % 2 else s for i, s in enumerate(seqs)]
    got, _ = T().twopaco_build_ex(low, 13, 1 << 16, 1)
    _eq(got, O.junctions(seqs, 13))


def test_unaligned_device_input():
    import torch
    seqs = _named("plain_single", 0.01)
    bases, off = G.concat(seqs)
    k, bits = 21, 1 << 18
    raw = torch.zeros(bases.size + 64, dtype=torch.uint8, device="cuda")
    raw[3:3 + bases.size] = torch.from_numpy(bases).cuda()
    d_off = torch.from_numpy(off.view(np.int64)).cuda()
    ws = T().twopaco_workspace_size(bases.size, len(seqs), k, bits, 1)
    wst = torch.empty(ws + 256, dtype=torch.uint8, device="cuda")
    wsp = (wst.data_ptr() + 255) // 256 * 256
    out_off = torch.zeros(len(seqs) + 1, dtype=torch.int64, device="cuda")
    out_pos = torch.zeros(bases.size, dtype=torch.int64, device="cuda")
    T().twopaco_run_device(raw.data_ptr() + 3, d_off.data_ptr(), len(seqs), bases.size, k, bits, 1,
                           None, wsp, ws, out_off.data_ptr(), out_pos.data_ptr(), bases.size)
    T().twopaco_read_stats(wsp)
    o = out_off.cpu().numpy()
    p = out_pos.cpu().numpy()
    _eq([p[o[t]:o[t + 1]] for t in range(len(seqs))], O.junctions((bases, off), k))


def test_bad_base_is_reported():
    seqs = ["ACGTACGTTTGACCA", "ACGTNACGT", "ACGTX"]
    with pytest.raises(T().TwopacoError) as e:
        T().twopaco_build_ex(seqs, 5, 1 << 12, 1)
    assert e.value.code == T().EBADBASE
    bases, off = G.concat([np.frombuffer(s.encode(), np.uint8) for s in seqs])
    run = T().DeviceBuild(bases, off, 5, 1 << 12, 1)
    run.run()
    st = run.stats(check=False)
    assert st["rc"] == T().EBADBASE and st["bad_base_index"] == 15 + 4


def test_table_overflow_is_reported_and_recovered():
    seqs = _named("plain_single", 0.05)
    bases, off = G.concat(seqs)
    opts = T().Options(hashes=3, table_slots=1024)
    run = T().DeviceBuild(bases, off, 25, 1 << 18, 1, opts)
    run.run()
    st = run.stats(check=False)
    assert st["rc"] == T().EOVERFLOW and st["overflow"]
    got, st = T().twopaco_build_ex(seqs, 25, 1 << 18, 1, opts)  # grows the table and reruns
    _eq(got, O.junctions((bases, off), 25))
    assert st["table_slots"] > 1024


def test_non_default_stream_and_repeat():
    import torch
    seqs = _named("plain_single", 0.05)
    bases, off = G.concat(seqs)
    want = O.junctions((bases, off), 25)
    run = T().DeviceBuild(bases, off, 25, 1 << 20, 2, T().Options(hashes=4, partition_bins=256))
    s = torch.cuda.Stream()
    for _ in range(3):
        run.run(stream=s)
    _eq(run.result(stream=s), want)


def test_candidate_list_overflow_falls_back_to_bitmap_walk():
    """A candidate list too short for the round: pass 2 walks C_temp instead."""
    seqs = _named("plain_single", 0.1)
    bases, off = G.concat(seqs)
    want = O.junctions((bases, off), 25)
    for recs in (1, 1000, 100000):
        run = T().DeviceBuild(bases, off, 25, 1 << 18, 1,
                              T().Options(hashes=3, candidate_records=recs))
        run.run()
        _eq(run.result(), want)
    got, _ = T().twopaco_build_ex(seqs, 25, 1 << 18, 2,
                                  T().Options(hashes=3, candidate_records=500, partition_bins=64))
    _eq(got, want)


def test_context_reuse_across_sizes_and_k():
    """One context, builds of growing and shrinking inputs: every result exact."""
    ctx = T().Context()
    cases = [("plain_single", 0.02, 25), ("plain_single", 0.25, 25), ("batched_set", 0.01, 31),
             ("plain_single", 0.02, 63), ("plain_single", 0.05, 17)]
    for name, scale, k in cases:
        seqs = _named(name, scale)
        got, st = ctx.build(seqs, k, 1 << 20, 1, T().Options(hashes=4))
        _eq(got, O.junctions(G.concat(seqs), k))
        assert st["pass2_marks"] == sum(g.size for g in got)
    # views into the context's buffers: valid until the next call
    seqs = _named("plain_single", 0.02)
    view, _ = ctx.build(seqs, 25, 1 << 20, 1, copy=False)
    _eq(view, O.junctions(G.concat(seqs), 25))
    with pytest.raises(T().TwopacoError) as e:
        ctx.build(["ACGTNNACGT"], 3, 1 << 12, 1)
    assert e.value.code == T().EBADBASE
    got, _ = ctx.build(seqs, 25, 1 << 20, 2, T().Options(partition_bins=256))
    _eq(got, O.junctions(G.concat(seqs), 25))
    ctx.close()


@pytest.mark.parametrize("name,scale,k,both", [("plain_single", 0.05, 25, True),
                                                ("batched_set", 0.01, 31, True),
                                                ("plain_single", 0.02, 63, True),
                                                ("plain_single", 0.02, 21, False)])
def test_edges_match_oracle(name, scale, k, both):
    """Compacted-graph edges (consecutive junction pairs) against the oracle, field by field."""
    seqs = _named(name, scale)
    ctx = T().Context()
    ctx.build(seqs, k, 1 << 20, 1, T().Options(hashes=4, both_strands=both))
    off, got = ctx.edges()
    want = O.edges(G.concat(seqs), k, both_strands=both)
    assert np.array_equal(np.diff(off), want["per_string"])
    for f in ("from_hi", "from_lo", "to_hi", "to_lo", "start", "length", "from_rc", "to_rc"):
        assert np.array_equal(got[f].astype(np.uint64), want[f].astype(np.uint64)), f
    ctx.close()


def test_edges_fig1_and_tiny_strings():
    ctx = T().Context()
    ctx.build(["TGGCACGTC", "TGGCACTTC", "A", ""], 2, 1 << 12, 1, T().Options(both_strands=False))
    off, e = ctx.edges()
    assert list(np.diff(off)) == [2, 2, 0, 0]
    assert list(e["length"]) == [4, 3, 4, 3]
    ctx.close()


def test_captured_run_replays_exactly():
    """A run captured as a CUDA graph: replays, and replays after rewriting the input in place."""
    import torch
    seqs_a = _named("plain_single", 0.05)
    bases_a, off = G.concat(seqs_a)
    # a second input of identical string lengths: the same strings, reverse-complemented
    comp = np.frombuffer(b"TGCA", np.uint8)
    code = {65: 0, 67: 1, 71: 2, 84: 3}
    seqs_b = [comp[np.array([code[int(c)] for c in s[::-1]])] for s in seqs_a]
    bases_b, off_b = G.concat(seqs_b)
    assert np.array_equal(off, off_b)
    run = T().DeviceBuild(bases_a, off, 25, 1 << 20, 2, T().Options(hashes=4, partition_bins=256))
    before = T().twopaco_kernel_launches()
    run.capture()
    assert T().twopaco_kernel_launches() == before, "capturing launches nothing"
    for _ in range(3):
        run.run()
    per_replay = (T().twopaco_kernel_launches() - before) // 3
    assert per_replay > 0
    _eq(run.result(), O.junctions((bases_a, off), 25))
    run.bases.copy_(torch.from_numpy(bases_b).cuda())  # same buffer, new content
    run.run()
    _eq(run.result(), O.junctions((bases_b, off), 25))
    run.release_plan()


def test_captured_run_profiles_every_replay():
    seqs = _named("plain_single", 0.02)
    bases, off = G.concat(seqs)
    run = T().DeviceBuild(bases, off, 25, 1 << 20, 1, T().Options(hashes=4))
    T().twopaco_profile_enable(True)
    try:
        run.capture()
        for _ in range(2):
            run.run()
            prof = T().twopaco_profile_kernels()
            assert prof["pass1_probe"]["ms"] > 0 and prof["pass1_insert"]["launches"] == 1
    finally:
        T().twopaco_profile_enable(False)
        run.release_plan()
    _eq(run.result(), O.junctions((bases, off), 25))


def test_bounded_wait_gives_up_and_the_context_survives():
    """A device wait on a flag that nothing sets ends with ETIMEOUT, not a hang, and the
    context stays usable: the failure path of the emit's look-back, made to happen."""
    import time
    t0 = time.time()
    assert T().twopaco_selftest_bounded_wait() == T().ETIMEOUT
    assert time.time() - t0 < 60
    got, _ = T().twopaco_build_ex(["TGGCACGTC", "TGGCACTTC"], 2, 1 << 12, 1,
                                  T().Options(both_strands=False))
    _eq(got, [[0, 4, 7], [0, 4, 7]])


# --- one launch per string (the per-genome baseline of the batched launch) ---------

@pytest.mark.parametrize("k,rounds,partial", [(25, 1, False), (31, 3, False), (63, 1, False),
                                              (25, 2, True), (100, 2, False)])
def test_per_string_launches_give_the_same_build(k, rounds, partial):
    """Every loop launched once per genome (tiles owned by the genome holding their first
    position, pass 2 over C_temp): the same junctions, C_temp and counters as the joint
    launch -- and the oracle's junctions."""
    seqs = _named("batched_set", 0.02)
    bases, off = G.concat(seqs)
    base = dict(hashes=4, partition_bins=256, partial=partial)
    joint = T().DeviceBuild(bases, off, k, 1 << 22, rounds, T().Options(**base))
    joint.run()
    per = T().DeviceBuild(bases, off, k, 1 << 22, rounds, T().Options(per_string_launches=True, **base))
    n0 = T().twopaco_kernel_launches()
    per.run()
    launched = T().twopaco_kernel_launches() - n0
    a, b = joint.result(), per.result()
    _eq(b, a)
    if not partial:
        _eq(b, _oracle_named("batched_set", 0.02, k))
    sa, sb = joint.stats(), per.stats()
    if rounds == 1:  # (more rounds: two separate class cuts may differ)
        assert sa["pass1_marks"] == sb["pass1_marks"] and sa["positions"] == sb["positions"]
        m = int(off[-1])
        ca = _bits_to_marks(joint.state(T().STATE_CANDIDATES, (m + 31) // 32), m)
        cb = _bits_to_marks(per.state(T().STATE_CANDIDATES, (m + 31) // 32), m)
        assert np.array_equal(ca, cb)
    assert launched > 62 * (2 if partial else 4) * rounds
    with pytest.raises(T().TwopacoError) as e:
        per.capture()
    assert e.value.code == T().EINVAL


# --- first-pass inserts through region buckets ------------------------------------

@pytest.mark.parametrize("k,bits,h,rounds,extra", [
    (25, 1 << 20, 4, 1, {}), (31, 1 << 22, 3, 3, {}), (63, 1 << 20, 6, 1, {}), (100, 1 << 20, 4, 2, {}),
    (25, 1 << 20, 4, 1, {"per_string_launches": True}), (25, 1 << 20, 4, 2, {"partial": True}),
    (21, 1 << 20, 4, 1, {"wide_layout": 1}),
])
def test_bucketed_inserts_give_the_same_filter(k, bits, h, rounds, extra):
    """Every OR staged in the bucket of its filter region and applied region by region
    (forced on small filters): C_temp bit-exact with the oracle's first pass (one round)
    and with the direct inserts, and the oracle's junctions. A homopolymer string sends
    all its records to one bucket, which overflows into direct ORs."""
    seqs = [s for s in _named("plain_single", 0.05)] + [np.frombuffer(b"A" * 60000, np.uint8)]
    bases, off = G.concat(seqs)
    m = int(off[-1])
    base = dict(hashes=h, partition_bins=256, **extra)
    a = T().DeviceBuild(bases, off, k, bits, rounds, T().Options(bucket_inserts=2, **base))
    b = T().DeviceBuild(bases, off, k, bits, rounds, T().Options(bucket_inserts=1, **base))
    assert b.ws_bytes > a.ws_bytes  # the buckets
    a.run()
    b.run()
    _eq(b.result(), a.result())
    if not extra.get("partial"):
        _eq(b.result(), O.junctions((bases, off), k))
    if rounds == 1:
        ca = _bits_to_marks(a.state(T().STATE_CANDIDATES, (m + 31) // 32), m)
        cb = _bits_to_marks(b.state(T().STATE_CANDIDATES, (m + 31) // 32), m)
        assert np.array_equal(ca, cb)
        if not extra.get("wide_layout"):
            marks, _, _, kept = O.pass1_marks((bases, off), k, bits, h)
            assert np.array_equal(cb, marks) and b.stats()["pass1_marks"] == kept


def test_bucketed_inserts_on_a_filter_beyond_l2():
    """A 2^30-bit (128 MiB) filter: with buckets (4 regions of 32 MiB) the same C_temp and
    junctions. Left automatic on this small input it stays direct (too few ORs per filter
    sector); the full-size 62-genome set takes the buckets automatically (its parity test
    is in test_gpu_timed_configs)."""
    seqs = _named("batched_set", 0.02)
    bases, off = G.concat(seqs)
    auto = T().DeviceBuild(bases, off, 25, 1 << 30, 1, T().Options(hashes=4))
    direct = T().DeviceBuild(bases, off, 25, 1 << 30, 1, T().Options(hashes=4, bucket_inserts=2))
    forced = T().DeviceBuild(bases, off, 25, 1 << 30, 1, T().Options(hashes=4, bucket_inserts=1))
    assert auto.ws_bytes == direct.ws_bytes < forced.ws_bytes
    full = sum(x.size for x in _named("batched_set", 1.0))
    assert T().twopaco_workspace_size(full, 62, 25, 1 << 30, 1) > \
        T().twopaco_workspace_size(full, 62, 25, 1 << 30, 1, T().Options(bucket_inserts=2))
    forced.run()
    _eq(forced.result(), _oracle_named("batched_set", 0.02, 25))
    m = int(off[-1])
    marks, _, _, kept = O.pass1_marks((bases, off), 25, 1 << 30, 4)
    assert np.array_equal(_bits_to_marks(forced.state(T().STATE_CANDIDATES, (m + 31) // 32), m), marks)


@pytest.mark.parametrize("shape,rounds", [(1, 1), (3, 1), (2, 3)])
def test_launch_shape_changes_nothing(shape, rounds):
    """Fewer resident blocks per SM in the pass kernels' grids: the same junctions."""
    seqs = _named("plain_single", 0.05)
    bases, off = G.concat(seqs)
    got, _ = T().twopaco_build_ex(seqs, 25, 1 << 20, rounds,
                                  T().Options(hashes=4, partition_bins=256, launch_blocks_per_sm=shape))
    _eq(got, O.junctions((bases, off), 25))
