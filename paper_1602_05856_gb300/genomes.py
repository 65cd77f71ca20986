"""Seeded synthetic genome sets shaped like the paper's workloads.

The paper measures on real assemblies (62 E. coli genomes, human assemblies,
UCSC primates; Results section, Tables 2-4) that are not available here.
These generators stand in for them: an ancestor is drawn at random, repeat
families are planted in it, and every genome is derived from it by point
substitutions, short indels, large deletions and structural variants
(inversions and transpositions).

This module holds no part of the junction method. It only draws bytes. Both
the CUDA path and the CPU oracle take its output as input. Every draw goes
through ``numpy.random.Generator(PCG64)`` built from a ``SeedSequence``, so
the same seed gives the same bytes on every platform numpy supports.

Sequences are ``numpy.uint8`` arrays of upper-case ASCII ``A C G T``.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence, Tuple

import numpy as np

_ACGT = np.frombuffer(b"ACGT", dtype=np.uint8).copy()
_CODE = np.full(256, 255, dtype=np.uint8)
for _i, _c in enumerate(b"ACGT"):
    _CODE[_c] = _i
_SWAP = np.zeros(256, dtype=np.uint8)
for _a, _b in zip(b"ACGT", b"TGCA"):
    _SWAP[_a] = _b


def random_bases(rng: np.random.Generator, n: int, gc: float = 0.5) -> np.ndarray:
    """``n`` i.i.d. bases; G and C each with probability ``gc / 2``."""
    at = (1.0 - gc) / 2.0
    idx = rng.choice(4, size=int(n), p=[at, gc / 2.0, gc / 2.0, at])
    return _ACGT[idx]


def substitute(rng: np.random.Generator, seq: np.ndarray, rate: float) -> np.ndarray:
    """Replace each base, with probability ``rate``, by one of the 3 others."""
    out = seq.copy()
    hit = np.flatnonzero(rng.random(seq.size) < rate)
    if hit.size:
        shift = rng.integers(1, 4, size=hit.size)
        out[hit] = _ACGT[(_CODE[seq[hit]].astype(np.int64) + shift) % 4]
    return out


def _splice(seq: np.ndarray, events: List[Tuple[int, int, np.ndarray]]) -> np.ndarray:
    """Apply (position, n_deleted, inserted) events given in ascending position."""
    pieces = []
    cursor = 0
    for pos, n_del, ins in events:
        if pos < cursor:
            continue
        pieces.append(seq[cursor:pos])
        if ins.size:
            pieces.append(ins)
        cursor = min(seq.size, pos + n_del)
    pieces.append(seq[cursor:])
    return np.concatenate(pieces) if pieces else seq.copy()


def indels(rng: np.random.Generator, seq: np.ndarray, rate: float,
           max_len: int = 10) -> np.ndarray:
    """Short insertions and deletions at ``rate`` per base.

    Half of the events insert, half delete; lengths are uniform in
    ``[1, max_len]``; inserted bases are uniform ACGT.
    """
    n_ev = int(rng.binomial(seq.size, rate))
    if n_ev == 0:
        return seq.copy()
    pos = np.sort(rng.integers(0, seq.size, size=n_ev))
    lens = rng.integers(1, max_len + 1, size=n_ev)
    is_ins = rng.random(n_ev) < 0.5
    ins_total = int(lens[is_ins].sum())
    ins_bases = random_bases(rng, ins_total)
    events = []
    o = 0
    for p, ln, ins in zip(pos.tolist(), lens.tolist(), is_ins.tolist()):
        if ins:
            events.append((p, 0, ins_bases[o:o + ln]))
            o += ln
        else:
            events.append((p, ln, ins_bases[:0]))
    return _splice(seq, events)


def plant_repeats(rng: np.random.Generator, seq: np.ndarray, family_len: int,
                  copies: int, divergence: float) -> np.ndarray:
    """Insert ``copies`` diverged copies of one random consensus at uniform positions."""
    consensus = random_bases(rng, family_len)
    pos = np.sort(rng.integers(0, seq.size + 1, size=copies))
    events = [(int(p), 0, substitute(rng, consensus, divergence)) for p in pos]
    return _splice(seq, events)


def reverse_strand(seq: np.ndarray) -> np.ndarray:
    """The other strand of ``seq`` read 5' to 3' (used for inversions)."""
    return _SWAP[seq[::-1]]


def structural_variants(rng: np.random.Generator, seq: np.ndarray, count: int,
                        min_len: int, max_len: int) -> np.ndarray:
    """``count`` inversions or transpositions (one or the other, even odds)."""
    out = seq
    for _ in range(count):
        ln = int(rng.integers(min_len, max_len + 1))
        if ln >= out.size:
            continue
        start = int(rng.integers(0, out.size - ln + 1))
        seg = out[start:start + ln]
        if rng.random() < 0.5:
            out = np.concatenate([out[:start], reverse_strand(seg), out[start + ln:]])
        else:
            rest = np.concatenate([out[:start], out[start + ln:]])
            dst = int(rng.integers(0, rest.size + 1))
            out = np.concatenate([rest[:dst], seg, rest[dst:]])
    return out


def trim_to(rng: np.random.Generator, seq: np.ndarray, target: int,
            blocks: int = 4) -> np.ndarray:
    """Remove ``len - target`` bases as ``blocks`` large deletions at random places."""
    excess = seq.size - int(target)
    if excess <= 0:
        return seq.copy()
    cuts = np.sort(rng.integers(0, excess + 1, size=blocks - 1))
    sizes = np.diff(np.concatenate([[0], cuts, [excess]]))
    out = seq
    for sz in sizes.tolist():
        if sz <= 0:
            continue
        start = int(rng.integers(0, out.size - sz + 1))
        out = np.concatenate([out[:start], out[start + sz:]])
    return out


@dataclass(frozen=True)
class GenomeSetSpec:
    """Recipe of one synthetic genome set (all rates are per base)."""
    n_genomes: int
    ancestor_len: int
    len_lo: int
    len_hi: int
    gc: float
    snp: float
    indel: float
    indel_max: int
    sv_count: int
    sv_min: int
    sv_max: int
    repeat_len: int
    repeat_copies: int
    repeat_div: float


# Four related 1 Mbp genomes: 940 kbp uniform ancestor + 200 x 300 bp repeat
# copies at 5% divergence, star tree, 0.5% SNPs, 0.05% indels of 1-10 bp.
PLAIN_SINGLE = GenomeSetSpec(4, 940_000, 1_000_000, 1_000_000, 0.5, 0.005, 0.0005, 10,
                             0, 0, 0, 300, 200, 0.05)
# Seven bacterial-size genomes, 4.6-5.6 Mbp, from a 50% GC ancestor with a
# 1.5 kbp x 30 repeat family; 1% SNPs, 0.1% indels, 20 SVs of 1-50 kbp.
BACTERIAL_SET = GenomeSetSpec(7, 5_555_000, 4_600_000, 5_600_000, 0.5, 0.01, 0.001, 10,
                              20, 1_000, 50_000, 1_500, 30, 0.02)
# 62 genomes of 4.5-5.5 Mbp (about 310 Mbp, the size of the 62 E. coli set).
BATCHED_SET = GenomeSetSpec(62, 5_455_000, 4_500_000, 5_500_000, 0.5, 0.01, 0.001, 10,
                            20, 1_000, 50_000, 1_500, 30, 0.02)

SEEDS = {"plain_single": 1602, "bacterial_set": 1603, "batched_set": 1604}
SPECS = {"plain_single": PLAIN_SINGLE, "bacterial_set": BACTERIAL_SET,
         "batched_set": BATCHED_SET}


def genome_set(spec: GenomeSetSpec, seed: int) -> List[np.ndarray]:
    """Draw one genome set: an ancestor, then ``n_genomes`` independent descendants."""
    ss = np.random.SeedSequence(seed)
    anc_seq, *child_seqs = ss.spawn(1 + spec.n_genomes)
    rng = np.random.Generator(np.random.PCG64(anc_seq))
    anc = random_bases(rng, spec.ancestor_len, spec.gc)
    if spec.repeat_copies:
        anc = plant_repeats(rng, anc, spec.repeat_len, spec.repeat_copies, spec.repeat_div)
    genomes = []
    for cs in child_seqs:
        r = np.random.Generator(np.random.PCG64(cs))
        g = anc
        if spec.len_hi > spec.len_lo or anc.size > spec.len_hi:
            g = trim_to(r, g, int(r.integers(spec.len_lo, spec.len_hi + 1)))
        g = substitute(r, g, spec.snp)
        g = indels(r, g, spec.indel, spec.indel_max)
        if spec.sv_count:
            g = structural_variants(r, g, spec.sv_count, spec.sv_min, spec.sv_max)
        genomes.append(np.ascontiguousarray(g, dtype=np.uint8))
    return genomes


def named_set(name: str, scale: float = 1.0) -> List[np.ndarray]:
    """One of the named workloads; ``scale`` < 1 shrinks every length (for tests)."""
    spec = SPECS[name]
    if scale != 1.0:
        def s(x: int) -> int:
            return max(1, int(round(x * scale)))
        spec = GenomeSetSpec(spec.n_genomes, s(spec.ancestor_len), s(spec.len_lo),
                             s(spec.len_hi), spec.gc, spec.snp, spec.indel, spec.indel_max,
                             spec.sv_count, max(1, s(spec.sv_min)), max(1, s(spec.sv_max)),
                             spec.repeat_len, spec.repeat_copies, spec.repeat_div)
    return genome_set(spec, SEEDS[name])


def random_strings(seed: int, n: int, min_len: int, max_len: int,
                   alphabet: bytes = b"ACGT") -> List[np.ndarray]:
    """Independent uniform strings (tiny brute-force cases)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    return [alpha[rng.integers(0, alpha.size, size=int(rng.integers(min_len, max_len + 1)))]
            for _ in range(n)]


def concat(seqs: Sequence[np.ndarray]) -> Tuple[np.ndarray, np.ndarray]:
    """Concatenate sequences; return (bytes, offsets) with ``offsets[i]`` the start of i."""
    lens = np.array([s.size for s in seqs], dtype=np.uint64)
    offsets = np.zeros(len(seqs) + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:])
    buf = np.concatenate(list(seqs)) if seqs else np.zeros(0, np.uint8)
    return np.ascontiguousarray(buf, dtype=np.uint8), offsets


def plant_n_runs(seed: int, seqs: Sequence[np.ndarray], runs_per_mbp: float = 50.0,
                 max_len: int = 5000, lower_frac: float = 0.1,
                 ends: bool = True) -> List[np.ndarray]:
    """Copies of ``seqs`` with runs of N written over them, like assembly gaps.

    Per string about ``runs_per_mbp`` runs per Mbp (at least one), at uniform
    places, of log-uniform length in [1, max_len]; a ``lower_frac`` share is
    written as 'n'. With ``ends`` every third string also starts or ends in N.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for t, s in enumerate(seqs):
        s = np.array(s, dtype=np.uint8, copy=True)
        if s.size:
            n_runs = max(1, int(rng.poisson(runs_per_mbp * s.size / 1e6)))
            for _ in range(n_runs):
                ln = int(np.exp(rng.uniform(0.0, np.log(max_len + 1))))
                a = int(rng.integers(0, s.size))
                s[a:a + ln] = ord("n") if rng.uniform() < lower_frac else ord("N")
            if ends and t % 3 == 0:
                ln = int(rng.integers(1, 40))
                if rng.integers(0, 2):
                    s[:ln] = ord("N")
                else:
                    s[-ln:] = ord("N")
        out.append(s)
    return out


def mammal_slice(seed: int = 1605, genome_len: int = 1_000_000, leaves: int = 8,
                 repeat_share: float = 0.45) -> List[np.ndarray]:
    """A slice of the mammal-scale configuration: ``leaves`` genomes of about
    ``genome_len`` bases at the leaves of a seeded random binary tree.

    The ancestor is ``repeat_share`` repeats: copies of a 300 bp family at
    10-15% divergence each and of a 6 kbp family, 20 copies of the short one
    per copy of the long one, the counts scaled to reach the share (the
    configuration's literal counts give 20%, its stated share 45%). Every tree
    edge mutates with SNPs and 1-10 bp indels at 10:1 and a few inversions or
    transpositions, at per-edge rates drawn so that two leaves differ by about
    1-8%. Full size would be 8 x 3 Gbp; the slice keeps the structure.
    """
    ss = np.random.SeedSequence(seed)
    anc_ss, tree_ss = ss.spawn(2)
    rng = np.random.Generator(np.random.PCG64(anc_ss))
    anc = random_bases(rng, genome_len, 0.41)
    unit = int(round(repeat_share * genome_len / (20 * 300 + 6_000)))  # copies of the 6 kbp family
    long_cons, short_cons = random_bases(rng, 6_000), random_bases(rng, 300)
    for cons, copies in ((long_cons, unit), (short_cons, 20 * unit)):
        for _ in range(copies):  # written over the ancestor: its length stays genome_len
            c = substitute(rng, cons, float(rng.uniform(0.10, 0.15)))
            at = int(rng.integers(0, max(1, anc.size - c.size)))
            anc[at:at + c.size] = c[: anc.size - at]
    # a random binary tree with `leaves` leaves: split the leaf set at random, recursively
    r = np.random.Generator(np.random.PCG64(tree_ss))

    def evolve(seq: np.ndarray, n: int) -> List[np.ndarray]:
        if n == 1:
            return [np.ascontiguousarray(seq, dtype=np.uint8)]
        left = int(r.integers(1, n))
        out = []
        for part in (left, n - left):
            rate = float(r.uniform(0.002, 0.012))  # per-edge divergence
            child = substitute(r, seq, rate * 10 / 11)
            child = indels(r, child, rate / 11, 10)
            child = structural_variants(r, child, int(r.integers(0, 3)), 1_000, 20_000)
            out += evolve(child, part)
        return out

    return evolve(anc, leaves)
