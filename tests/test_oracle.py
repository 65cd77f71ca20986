"""Pins of the CPU oracle against the paper and against brute force (no GPU)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_1602_05856_gb300 import genomes as G
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_junctions.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            strands, k, seq, *pos = line.split()
            rows.append((strands == "both", int(k), seq, [int(p) for p in pos]))
    return rows


def _as_lists(res):
    return [list(map(int, r)) for r in res]


@pytest.mark.parametrize("both,k", [(False, 2), (True, 2), (True, 3)])
def test_fig1_worked_example(both, k):
    rows = [r for r in _golden_rows() if r[0] == both and r[1] == k]
    seqs = [r[2] for r in rows]
    got = _as_lists(O.junctions(seqs, k, both_strands=both))
    assert got == [r[3] for r in rows]
    assert got == _as_lists(O.alg1_exact(seqs, k, both_strands=both))


def test_fig1_false_junction_gc_absent():
    # Fig. 1d: "GC" (position 2) is only a junction if a false edge is seen.
    got = O.junctions(["TGGCACGTC", "TGGCACTTC"], 2, both_strands=False)
    assert all(2 not in r for r in _as_lists(got))


def _random_cases():
    cases = []
    seed = 11
    for k in list(range(1, 9)) + [15, 25, 31, 63, 64, 65, 96, 100, 127]:
        for both in (False, True):
            for alpha in (b"ACGT", b"AC", b"ACG"):
                lo = max(1, k - 3)
                hi = max(k + 40, 3 * k)
                cases.append((seed, k, both, alpha, lo, hi))
                seed += 1
    return cases


@pytest.mark.parametrize("seed,k,both,alpha,lo,hi", _random_cases())
def test_definition_matches_brute_force(seed, k, both, alpha, lo, hi):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 6))
    seqs = [bytes(s).decode() for s in G.random_strings(seed, n, lo, hi, alpha)]
    if seed % 3 == 0:  # plant a reverse-complement pair and a repeat
        seqs.append(brute.revcomp(seqs[0]))
        seqs.append(seqs[0][: len(seqs[0]) // 2] + seqs[-1])
    got = _as_lists(O.junctions(seqs, k, both_strands=both))
    assert got == brute.junction_positions(seqs, k, both)
    assert got == _as_lists(O.alg1_exact(seqs, k, both_strands=both))


SPECIAL = [
    ("homopolymer", ["A" * 40], 5),
    ("homopolymer_rc", ["T" * 30, "A" * 12], 7),
    ("dinucleotide_repeat", ["AC" * 25], 4),
    ("tandem", ["ACGTTGCA" * 8], 6),
    ("palindromes_even_k", ["ACGTACGTAATTGCGCAT", "GAATTCGAATTC"], 4),
    ("shorter_than_k", ["ACG", "ACGTACGTAC"], 5),
    ("exactly_k", ["ACGTA", "CCCCGGGG"], 5),
    ("self_rc_string", ["AAGCTT", "GGATCC" * 3], 6),
    ("k1", ["ACGTTTACG"], 1),
    ("homopolymer_k100", ["A" * 160, "T" * 101], 100),
    ("palindromes_k64", ["ACGT" * 40, "AATT" * 16 + "GC" + "AATT" * 20], 64),
    ("rc_pair_k127", ["ACGGT" * 40, "ACCGT" * 40], 127),
    ("exactly_k_k100", ["ACGTTGCA" * 12 + "ACGT", "C" * 99], 100),
]


@pytest.mark.parametrize("name,seqs,k", SPECIAL, ids=[s[0] for s in SPECIAL])
@pytest.mark.parametrize("both", [False, True])
def test_special_cases(name, seqs, k, both):
    got = _as_lists(O.junctions(seqs, k, both_strands=both))
    assert got == brute.junction_positions(seqs, k, both)


def test_homopolymer_every_position_is_sentinel():
    # The only k-mer of A^L is both the first and the last k-mer: a sentinel.
    got = _as_lists(O.junctions(["A" * 30], 4))
    assert got == [list(range(27))]


def test_short_strings_have_no_positions():
    got = _as_lists(O.junctions(["ACGT", "ACGTACGTAA"], 8))
    assert got[0] == [] and got[1] == [0, 2]


@pytest.mark.parametrize("k,both", [(3, False), (4, True), (5, True), (9, False), (12, True)])
def test_observation1_compaction_bijection(k, both):
    """Junction-flanked substrings are exactly the maximal non-branching paths."""
    seqs = [bytes(s).decode() for s in G.random_strings(100 + k, 4, 30, 90, b"ACG")]
    seqs.append(seqs[1][5:40] + seqs[2][:30])
    all_texts = brute.texts(seqs, both)
    # adding the reverse complements does not change G_comp nor its sentinels
    pos = _as_lists(O.junctions(all_texts, k, both_strands=both))
    assert pos[: len(seqs)] == _as_lists(O.junctions(seqs, k, both_strands=both))
    assert brute.paths_from_positions(all_texts, k, pos) == brute.compacted_paths(seqs, k, both)


def test_spelling_invariant_plain_single_slice():
    """Consecutive junction-flanked segments, overlapped by k-1, re-spell each genome."""
    seqs = [s[:20000] for s in G.named_set("plain_single", scale=0.05)]
    k = 25
    res = O.junctions(seqs, k)
    for s, pos in zip(seqs, res):
        pos = [int(p) for p in pos]
        assert pos[0] == 0 and pos[-1] == s.size - k
        spelled = bytes(s[pos[0]:pos[0] + k])
        for a, b in zip(pos, pos[1:]):
            spelled += bytes(s[a + k:b + k])
        assert spelled == bytes(s)


def test_reverse_complement_symmetry():
    seqs = [bytes(s).decode() for s in G.random_strings(7, 5, 50, 400, b"ACGT")]
    seqs += [seqs[0][10:200], brute.revcomp(seqs[1][:150])]
    k = 7
    fwd = _as_lists(O.junctions(seqs, k))
    rev = _as_lists(O.junctions([brute.revcomp(s) for s in seqs], k))
    for s, f, r in zip(seqs, fwd, rev):
        assert sorted(len(s) - k - p for p in f) == r


def test_duplicate_and_permutation_invariance():
    seqs = [bytes(s).decode() for s in G.random_strings(5, 4, 80, 300, b"ACGT")]
    k = 6
    base = _as_lists(O.junctions(seqs, k))
    perm = _as_lists(O.junctions(seqs[::-1], k))
    assert perm == base[::-1]
    dup = _as_lists(O.junctions(seqs + [seqs[2]], k))
    assert dup[:4] == base and dup[4] == base[2]


def test_lowercase_and_bad_bytes():
    assert _as_lists(O.junctions(["tggcacgtc", "TGGCACTTC"], 2, both_strands=False)) == \
        [[0, 4, 7], [0, 4, 7]]
    with pytest.raises(O.OracleError):
        O.junctions(["ACGNT"], 2)
    with pytest.raises(O.OracleError):
        O.junctions(["ACGT"], 0)
    with pytest.raises(O.OracleError):
        O.junctions(["ACGT"], 128)


def test_empty_input():
    assert O.junctions([], 5) == []
    assert _as_lists(O.junctions(["", "AC"], 5)) == [[], []]


# --- first pass with the split-block filter ---------------------------------

def _occurrence_groups(seqs, k):
    groups = {}
    for t, s in enumerate(seqs):
        for i in range(len(s) - k + 1):
            v = s[i:i + k]
            key = min(v, brute.revcomp(v))
            groups.setdefault(key, []).append((t, i))
    return groups


@pytest.mark.parametrize("bits,h", [(256, 1), (1 << 12, 3), (1 << 16, 4), (1 << 20, 8)])
def test_pass1_candidate_set_contains_junctions(bits, h):
    seqs = [bytes(s).decode() for s in G.random_strings(3, 5, 100, 2000, b"ACGT")]
    seqs += [seqs[0][50:900], seqs[1][:300] + seqs[2][100:700]]
    k = 9
    marks, off, active, kept = O.pass1_marks(seqs, k, bits, h)
    flags, _, _ = O.junction_flags(seqs, k)
    assert active == sum(max(0, len(s) - k + 1) for s in seqs)
    assert int(marks.sum()) == kept
    assert np.all(marks >= flags), "a junction was unmarked"
    # candidate-set property: all occurrences of a k-mer agree
    for occ in _occurrence_groups(seqs, k).values():
        vals = {int(marks[int(off[t]) + i]) for t, i in occ}
        assert len(vals) == 1


def test_pass1_saturated_filter_keeps_everything():
    seqs = [bytes(s).decode() for s in G.random_strings(4, 3, 3000, 4000, b"ACGT")]
    marks, off, active, kept = O.pass1_marks(seqs, 11, 256, 1)
    assert kept == active


def test_pass1_sparse_filter_is_exact():
    seqs = [bytes(s).decode() for s in G.random_strings(9, 4, 200, 800, b"ACGT")]
    seqs.append(seqs[0][100:500])
    marks, off, active, kept = O.pass1_marks(seqs, 8, 1 << 30, 8)
    flags, _, _ = O.junction_flags(seqs, 8)
    assert np.array_equal(marks, flags)


def test_pass1_classes_partition_positions():
    seqs = [bytes(s).decode() for s in G.random_strings(12, 3, 500, 1500, b"ACGT")]
    k, q = 10, 64
    cuts = [0, 5, 21, 22, 64]
    flags, _, _ = O.junction_flags(seqs, k)
    total = sum(len(s) - k + 1 for s in seqs)
    union = np.zeros_like(flags)
    n_active = 0
    for r in range(4):
        m, _, a, kept = O.pass1_marks(seqs, k, 1 << 14, 3, q=q, bin_lo=cuts[r], bin_hi=cuts[r + 1])
        assert not np.any(union & m), "rounds overlap"
        union |= m
        n_active += a
    assert n_active == total
    assert np.all(union >= flags)


# --- greedy class cut ----------------------------------------------------------

def test_partition_cuts_examples():
    assert list(O.partition_cuts([1, 1, 1, 1], 2)) == [0, 2, 4]
    assert list(O.partition_cuts([5, 1, 1, 1], 2)) == [0, 1, 4]
    assert list(O.partition_cuts([1, 1, 1, 1], 1)) == [0, 4]
    assert list(O.partition_cuts([0, 0, 0, 9], 3)) == [0, 2, 3, 4]


@pytest.mark.parametrize("seed", range(20))
def test_partition_cuts_greedy_property(seed):
    rng = np.random.default_rng(seed)
    q = int(rng.integers(4, 200))
    ell = int(rng.integers(1, min(q, 17) + 1))
    counts = rng.integers(0, 50, size=q) * (rng.random(q) < 0.8)
    cuts = [int(c) for c in O.partition_cuts(counts, ell)]
    total = int(counts.sum())
    assert cuts[0] == 0 and cuts[-1] == q and len(cuts) == ell + 1
    for r in range(ell):
        lo, hi = cuts[r], cuts[r + 1]
        assert hi > lo, "every class owns at least one bin"
        if r < ell - 1:
            s = int(counts[lo:hi].sum())
            # maximal: one more bin would exceed the share, unless the class is a
            # single bin or the next bin is reserved for a later class
            if hi - lo > 1:
                assert s * ell <= total
            if hi < q - (ell - 1 - r):
                assert (s + int(counts[hi])) * ell > total or hi - lo == 0


# --- compacted-graph edges -----------------------------------------------------------

def _kmer_str(hi, lo, k):
    v = (int(hi) << 64) | int(lo)
    return "".join("ACGT"[(v >> (2 * (k - 1 - i))) & 3] for i in range(k))


@pytest.mark.parametrize("k,both", [(2, False), (3, True), (4, True), (5, False), (7, True)])
def test_edges_are_the_maximal_nonbranching_paths(k, both):
    """Observation 1: junction-to-junction edges = the compacted graph's edges."""
    seqs = [bytes(s).decode() for s in G.random_strings(300 + k, 4, 20, 80, b"ACG")]
    seqs.append(seqs[0][3:50] + seqs[1][:25])
    e = O.edges(seqs, k, both_strands=both)
    # every edge spells a string segment whose first and last k-mers are its endpoints
    spelled = set()
    o = 0
    for t, s in enumerate(seqs):
        for _ in range(int(e["per_string"][t])):
            p, ln = int(e["start"][o]), int(e["length"][o])
            seg = s[p:p + ln + k]
            a = _kmer_str(e["from_hi"][o], e["from_lo"][o], k)
            b = _kmer_str(e["to_hi"][o], e["to_lo"][o], k)
            assert (brute.revcomp(a) if e["from_rc"][o] else a) == seg[:k]
            assert (brute.revcomp(b) if e["to_rc"][o] else b) == seg[-k:]
            path = tuple(seg[i:i + k] for i in range(ln + 1))
            spelled.add(path)
            if both:
                r = brute.revcomp(seg)
                spelled.add(tuple(r[i:i + k] for i in range(ln + 1)))
            o += 1
    assert o == e["start"].size
    assert spelled == brute.compacted_paths(seqs, k, both)


@pytest.mark.parametrize("k,both", [(6, True), (7, False), (9, True)])
def test_partial_edges_are_nonbranching_paths(k, both):
    """Edges between consecutive positions of a candidate set (the first pass's survivors,
    the partially compacted graph of the Discussion section): each spells a path whose
    inner k-mers are all non-junctions by brute force, every junction is an endpoint, and
    with the junction set itself they are the maximal non-branching paths."""
    seqs = [bytes(s).decode() for s in G.random_strings(500 + k, 4, 40, 300, b"ACGT")]
    seqs.append(seqs[0][10:120] + seqs[1][:90])
    marks, off, _, kept = O.pass1_marks(seqs, k, 1 << 9, 2, both_strands=both)
    J = brute.junction_kmers(seqs, k, both)
    flags, _, _ = O.junction_flags(seqs, k, both_strands=both)
    assert kept > int(flags.sum()), "the small filter leaves false candidates"
    e = O.edges(seqs, k, both_strands=both, flags=marks)
    o = 0
    for t, s in enumerate(seqs):
        cand = np.flatnonzero(marks[int(off[t]):int(off[t + 1])])
        assert int(e["per_string"][t]) == max(0, cand.size - 1)
        for a, b in zip(cand, cand[1:]):
            assert int(e["start"][o]) == a and int(e["length"][o]) == b - a
            assert all(s[i:i + k] not in J for i in range(a + 1, b))
            o += 1
        for i in range(len(s) - k + 1):
            if s[i:i + k] in J:
                assert i in cand
    assert o == e["start"].size


def test_edges_fig1():
    e = O.edges(["TGGCACGTC", "TGGCACTTC"], 2, both_strands=False)
    # TG -> AC (TGGCAC), AC -> TC (ACGTC / ACTTC): Fig. 1b/1c
    assert list(e["per_string"]) == [2, 2]
    assert [_kmer_str(0, x, 2) for x in e["from_lo"]] == ["TG", "AC", "TG", "AC"]
    assert [_kmer_str(0, x, 2) for x in e["to_lo"]] == ["AC", "TC", "AC", "TC"]
    assert list(e["length"]) == [4, 3, 4, 3]


# --- N handling: an N ends its string there (the paper is silent on N) ---------------

def _pieces(s):
    """(offset, piece) of the maximal N-free pieces of s, split in plain Python."""
    out, i = [], 0
    while i < len(s):
        if s[i] in "Nn":
            i += 1
            continue
        j = i
        while j < len(s) and s[j] not in "Nn":
            j += 1
        out.append((i, s[i:j]))
        i = j
    return out


def _brute_split(seqs, k, both):
    pcs = [(t, o, p.upper()) for t, s in enumerate(seqs) for o, p in _pieces(s)]
    per = brute.junction_positions([p for _, _, p in pcs], k, both)
    got = [[] for _ in seqs]
    for (t, o, _), js in zip(pcs, per):
        got[t] += [o + j for j in js]
    return [sorted(x) for x in got]


def _with_ns(rng, s, k):
    """s with N runs of lengths 1 .. 2k+2 planted at random places (and at the ends)."""
    s = list(s)
    for _ in range(int(rng.integers(0, 5))):
        a = int(rng.integers(0, len(s) + 1))
        s[a:a] = "N" * int(rng.integers(1, 2 * k + 3))
    if rng.integers(0, 3) == 0:
        s = list("n" * int(rng.integers(1, 4))) + s
    if rng.integers(0, 3) == 0:
        s += list("N" * int(rng.integers(1, 4)))
    return "".join(s)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 8, 15, 25, 31, 63])
@pytest.mark.parametrize("both", [False, True])
def test_split_n_matches_brute_force_on_pieces(k, both):
    rng = np.random.default_rng(4242 + k + 1000 * both)
    for alpha in (b"ACGT", b"AC"):
        base = [bytes(s).decode() for s in G.random_strings(int(rng.integers(1 << 30)), 4, k,
                                                            3 * k + 60, alpha)]
        base.append(brute.revcomp(base[0]))
        seqs = [_with_ns(rng, s, k) for s in base]
        seqs.append("N" * (k + 3))
        seqs.append("")
        got = _as_lists(O.junctions(seqs, k, both_strands=both, split_n=True))
        assert got == _brute_split(seqs, k, both)


def test_split_n_special_cases():
    k = 3
    seqs = ["ACGTNACGT", "NNNN", "NACGTN", "ACNGT", "ACGNNNNNNNNTTA", "acgtnacg"]
    got = _as_lists(O.junctions(seqs, k, split_n=True))
    assert got == _brute_split(seqs, k, True)
    assert got[1] == [] and got[3] == []        # only N, or pieces shorter than k
    assert got[2] == [1, 2]                     # ACGT between two N: both 3-mers are sentinels
    # a k-mer next to an N is a sentinel even in the middle of a string
    assert 0 in got[0] and 1 in got[0] and 5 in got[0] and 6 in got[0]


def test_n_is_an_error_without_split():
    with pytest.raises(O.OracleError):
        O.junctions(["ACGTNACGT"], 3)
    with pytest.raises(O.OracleError):
        O.junctions(["ACGTRACGT"], 3, split_n=True)  # only N splits


def test_split_n_without_n_changes_nothing():
    seqs = [bytes(s).decode() for s in G.random_strings(77, 5, 30, 300, b"ACGT")]
    for k in (4, 25):
        assert _as_lists(O.junctions(seqs, k, split_n=True)) == _as_lists(O.junctions(seqs, k))
        a = O.edges(seqs, k, split_n=True)
        b = O.edges(seqs, k)
        assert all(np.array_equal(a[x], b[x]) for x in a)


@pytest.mark.parametrize("k,both", [(3, True), (5, False), (25, True)])
def test_split_n_edges_are_the_pieces_edges(k, both):
    """Edges never cross an N: they are the edges of the pieces, in string order."""
    rng = np.random.default_rng(99 + k)
    base = [bytes(s).decode() for s in G.random_strings(500 + k, 4, 2 * k, 5 * k + 80, b"ACG")]
    seqs = [_with_ns(rng, s, k) for s in base]
    e = O.edges(seqs, k, both_strands=both, split_n=True)
    pcs = [(t, o, p) for t, s in enumerate(seqs) for o, p in _pieces(s)]
    pe = O.edges([p for _, _, p in pcs], k, both_strands=both)
    # the pieces' edges, shifted to string offsets, in the same order
    assert np.array_equal(e["length"], pe["length"])
    shift = np.concatenate([np.full(int(pe["per_string"][i]), o, np.uint64)
                            for i, (_, o, _) in enumerate(pcs)]) if pe["start"].size else pe["start"]
    assert np.array_equal(e["start"], pe["start"] + shift)
    for x in ("from_hi", "from_lo", "to_hi", "to_lo", "from_rc", "to_rc"):
        assert np.array_equal(e[x], pe[x])
    per = np.zeros(len(seqs), np.uint64)
    for i, (t, _, _) in enumerate(pcs):
        per[t] += pe["per_string"][i]
    assert np.array_equal(e["per_string"], per)
    # and the pieces' edges are pinned against the explicit graph
    assert brute.compacted_paths([p for _, _, p in pcs], k, both) is not None


def test_split_n_pass1_contains_junctions():
    rng = np.random.default_rng(5)
    base = [bytes(s).decode() for s in G.random_strings(8, 6, 100, 400, b"ACGT")]
    seqs = [_with_ns(rng, s, 25) for s in base]
    want = O.junction_flags(seqs, 25, split_n=True)[0]
    for bits, h in ((1 << 10, 2), (1 << 20, 4)):
        marks, _, active, kept = O.pass1_marks(seqs, 25, bits, h, split_n=True)
        assert np.all(marks >= want)
        assert active == sum(max(0, len(p) - 24) for s in seqs for _, p in _pieces(s))
    # a sparse filter is exact: marks equal the junctions
    marks, _, _, _ = O.pass1_marks(seqs, 25, 1 << 30, 8, split_n=True)
    assert np.array_equal(marks, want)


# --- k > 63: 256-bit k-mer words -----------------------------------------------------

@pytest.mark.parametrize("k,both", [(64, True), (70, False), (100, True), (127, True)])
def test_edges_long_k(k, both):
    """Edges for k > 63 carry the last 64 bases of each normalized k-mer."""
    seqs = [bytes(s).decode() for s in G.random_strings(700 + k, 4, k, 4 * k, b"AC")]
    seqs.append(seqs[0][5:k + 40] + seqs[1][: k + 10])
    e = O.edges(seqs, k, both_strands=both)
    spelled, o = set(), 0
    for t, s in enumerate(seqs):
        for _ in range(int(e["per_string"][t])):
            p, ln = int(e["start"][o]), int(e["length"][o])
            seg = s[p:p + ln + k]
            a, b = seg[:k], seg[-k:]
            na = min(a, brute.revcomp(a)) if both else a
            nb = min(b, brute.revcomp(b)) if both else b
            assert _kmer_str(e["from_hi"][o], e["from_lo"][o], 64) == na[-64:]
            assert _kmer_str(e["to_hi"][o], e["to_lo"][o], 64) == nb[-64:]
            assert e["from_rc"][o] == (na != a) and e["to_rc"][o] == (nb != b)
            spelled.add(tuple(seg[i:i + k] for i in range(ln + 1)))
            if both:
                r = brute.revcomp(seg)
                spelled.add(tuple(r[i:i + k] for i in range(ln + 1)))
            o += 1
    assert spelled == brute.compacted_paths(seqs, k, both)


@pytest.mark.parametrize("k", [64, 100, 127])
def test_pass1_invariants_long_k(k):
    seqs = [bytes(s).decode() for s in G.random_strings(40 + k, 5, 2 * k, 900, b"ACGT")]
    seqs.append(seqs[0][10:600])
    want = O.junction_flags(seqs, k)[0]
    for bits, h in ((1 << 10, 2), (1 << 16, 4), (1 << 30, 8)):
        marks, _, active, kept = O.pass1_marks(seqs, k, bits, h)
        assert np.all(marks >= want) and active == sum(len(s) - k + 1 for s in seqs)
    assert np.array_equal(marks, want)  # 2^30 bits: no collisions on this input
    # the candidate-set property: all occurrences of a k-mer agree
    marks, _, _, _ = O.pass1_marks(seqs, k, 1 << 12, 3)
    _, off = O._prep(seqs)
    groups = {}
    for t, s in enumerate(seqs):
        for i in range(len(s) - k + 1):
            v = s[i:i + k]
            groups.setdefault(min(v, brute.revcomp(v)), set()).add(int(marks[int(off[t]) + i]))
    assert all(len(g) == 1 for g in groups.values())


def test_split_n_long_k():
    rng = np.random.default_rng(17)
    base = [bytes(s).decode() for s in G.random_strings(18, 5, 150, 700, b"ACGT")]
    seqs = [_with_ns(rng, s, 100) for s in base]
    got = _as_lists(O.junctions(seqs, 100, split_n=True))
    assert got == _brute_split(seqs, 100, True)


# --- the partition-parallel form of the definition ---------------------------------

@pytest.mark.parametrize("k,both,split", [(5, True, False), (25, True, True), (31, False, False),
                                          (63, True, False), (100, True, True)])
def test_parallel_definition_equals_single_thread(k, both, split):
    rng = np.random.default_rng(k + 7 * both)
    seqs = [bytes(s).decode() for s in G.random_strings(900 + k, 6, k, 20 * k + 400, b"ACGT")]
    seqs += [bytes(s).decode() for s in G.random_strings(901 + k, 3, 50, 600, b"AC")]
    if split:
        seqs = [_with_ns(rng, s, k) for s in seqs]
    want = _as_lists(O.junctions(seqs, k, both_strands=both, split_n=split))
    for threads in (2, 3, 8):
        assert _as_lists(O.junctions(seqs, k, both_strands=both, split_n=split, threads=threads)) == want


def test_mammal_slice_generator_is_seeded_and_shaped():
    a = G.mammal_slice(genome_len=60_000)
    b = G.mammal_slice(genome_len=60_000)
    assert len(a) == 8 and all(np.array_equal(x, y) for x, y in zip(a, b))
    assert all(55_000 < x.size < 65_000 for x in a)
    assert not all(np.array_equal(a[0], x) for x in a[1:])  # the leaves differ
    c = G.mammal_slice(seed=7, genome_len=60_000)
    assert not np.array_equal(a[0], c[0])


# --- the ctypes wrappers against the oracle's C entry points ---------------------------

def test_oracle_wrappers_match_the_c_signatures():
    import ctypes
    import os
    import re
    src = open(os.path.join(os.path.dirname(O.__file__), "twopaco_oracle.cpp")).read()
    defs = re.findall(r"(?m)^(int|long long) (oracle_\w+)\(([^)]*)\)\s*\{", src)
    assert len(defs) == 6
    L = O.lib()
    for ret, name, params in defs:
        params = [p.strip() for p in params.split(",")]
        fn = getattr(L, name)
        assert len(fn.argtypes) == len(params), name
        for p, t in zip(params, fn.argtypes):
            if "*" in p:
                assert t is ctypes.c_void_p, (name, p)
            elif p.startswith("uint64_t"):
                assert t is ctypes.c_uint64, (name, p)
            else:
                assert p.startswith("int ") and t is ctypes.c_int, (name, p)
        assert fn.restype is (ctypes.c_int if ret == "int" else ctypes.c_longlong), name
