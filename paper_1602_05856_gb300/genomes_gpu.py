"""Seeded synthetic genome sets drawn on the GPU, for inputs too large to draw on the host.

The mammal-scale configuration -- 8 genomes of 3 Gbp at the leaves of a
random binary tree over an ancestor that is 45% repeats -- stands in for the
paper's 8 primates (Results section, Tables 3-4: 24.5 G positions). Drawing
24 Gbp with numpy on the host takes minutes and tens of GB of temporaries,
so this module draws the same recipe with PyTorch on the device, chunk by
chunk:

* ancestor: uniform bases at 41% GC;
* repeats written over it, at non-overlapping places: copies of a 6 kbp
  family and, 20 per long copy, of a 300 bp family, each copy with its own
  divergence drawn in [10%, 15%], the counts scaled so that the copies cover
  ``repeat_share`` of the ancestor (the configuration's literal counts,
  1e6 x 300 bp + 5e4 x 6 kbp, cover 20% of 3 Gbp; its stated share is 45%);
* a random binary tree with ``leaves`` leaves (split the leaf set at a
  uniform point, recursively); every edge draws a divergence in
  [0.2%, 1.2%] and applies it as SNPs and 1-10 bp indels at 10:1 (half
  insertions) plus 0-2 inversions or transpositions of 1-20 kbp, so that two
  leaves differ by about 1-8%.

It holds no part of the junction method: it only draws bytes (upper-case
ASCII A C G T). Every draw comes from one ``torch.Generator`` on the device
and one numpy ``PCG64`` on the host (tree shape, rates, event counts), both
seeded, so a seed gives the same bytes on the same GPU model and PyTorch
build. ``mammal_set(genome_len=...)`` at a smaller length draws a slice of
the same recipe, which the tests compare with the CPU oracle.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

CHUNK = 1 << 28  # bases per chunk of the per-base draws (bounds the temporaries)
_A, _C, _G, _T = 65, 67, 71, 84


def _torch():
    import torch
    return torch


def _random_bases(gen, n: int, gc: float, device):
    """n i.i.d. bases; C and G each with probability about gc / 2 (in 256ths)."""
    torch = _torch()
    out = torch.empty(n, dtype=torch.uint8, device=device)
    c = int(round(gc * 128))
    g = int(round(gc * 256)) - c
    a = (256 - c - g) // 2
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        b = torch.randint(0, 256, (e - s,), dtype=torch.uint8, generator=gen, device=device)
        o = torch.full((e - s,), _T, dtype=torch.uint8, device=device)
        o[b < c + g + a] = _A
        o[b < c + g] = _G
        o[b < c] = _C
        out[s:e] = o
    return out


def _codes(x):
    """A C G T -> 0 1 2 3 (int64)."""
    return (x == _C).long() + 2 * (x == _G).long() + 3 * (x == _T).long()


def _substitute(gen, seq, rate: float):
    """Each base, with probability rate, becomes one of the three others (in place)."""
    torch = _torch()
    lut = torch.tensor([_A, _C, _G, _T], dtype=torch.uint8, device=seq.device)
    for s in range(0, seq.numel(), CHUNK):
        e = min(seq.numel(), s + CHUNK)
        hit = torch.nonzero(torch.rand(e - s, generator=gen, device=seq.device) < rate).squeeze(1) + s
        if hit.numel():
            shift = torch.randint(1, 4, (hit.numel(),), generator=gen, device=seq.device)
            seq[hit] = lut[(_codes(seq[hit]) + shift) % 4]
    return seq


def _substitute_rows(gen, rows, rates):
    """Row i of a (copies x length) block mutated at rates[i] (in place)."""
    torch = _torch()
    lut = torch.tensor([_A, _C, _G, _T], dtype=torch.uint8, device=rows.device)
    step = max(1, CHUNK // rows.shape[1])
    for s in range(0, rows.shape[0], step):
        blk = rows[s:s + step]
        hit = torch.rand(blk.shape, generator=gen, device=rows.device) < rates[s:s + step, None]
        shift = torch.randint(1, 4, blk.shape, generator=gen, device=rows.device)
        blk[hit] = lut[(_codes(blk) + shift) % 4][hit]
    return rows


def _indels(gen, rng: np.random.Generator, seq, rate: float, max_len: int = 10):
    """Short insertions and deletions at rate per base (half each, lengths 1..max_len,
    inserted bases uniform), applied chunk by chunk."""
    torch = _torch()
    dev = seq.device
    out = []
    for s in range(0, seq.numel(), CHUNK):
        e = min(seq.numel(), s + CHUNK)
        n = e - s
        src = seq[s:e]
        n_ev = int(rng.binomial(n, rate))
        if n_ev == 0:
            out.append(src.clone())
            continue
        pos = torch.sort(torch.randint(0, n, (n_ev,), generator=gen, device=dev)).values
        lens = torch.randint(1, max_len + 1, (n_ev,), generator=gen, device=dev)
        ins = torch.rand(n_ev, generator=gen, device=dev) < 0.5
        # deleted bases: +1 at a deletion's start, -1 after its end, summed along
        diff = torch.zeros(n + 1, dtype=torch.int32, device=dev)
        dpos, dlen = pos[~ins], lens[~ins]
        diff.index_add_(0, dpos, torch.ones_like(dpos, dtype=torch.int32))
        diff.index_add_(0, torch.clamp(dpos + dlen, max=n), -torch.ones_like(dpos, dtype=torch.int32))
        keep = torch.cumsum(diff, 0)[:n] == 0
        # inserted bases go before their position
        ins_len = torch.zeros(n, dtype=torch.int64, device=dev)
        ins_len.index_add_(0, pos[ins], lens[ins])
        count = keep.long() + ins_len
        start = torch.cumsum(count, 0) - count
        total = int(count.sum().item())
        o = _random_bases(gen, total, 0.5, dev)
        o[(start + ins_len)[keep]] = src[keep]
        out.append(o)
    return torch.cat(out)


_COMP = None


def _reverse_strand(x):
    torch = _torch()
    global _COMP
    if _COMP is None or _COMP.device != x.device:
        c = torch.zeros(256, dtype=torch.uint8)
        for a, b in zip(b"ACGT", b"TGCA"):
            c[a] = b
        _COMP = c.to(x.device)
    return _COMP[torch.flip(x, [0]).long()]


def _structural(gen, rng: np.random.Generator, seq, count: int, lo: int, hi: int):
    """count inversions or transpositions (even odds) of lo..hi bases."""
    torch = _torch()
    for _ in range(count):
        ln = int(rng.integers(lo, hi + 1))
        if ln >= seq.numel():
            continue
        a = int(rng.integers(0, seq.numel() - ln + 1))
        if rng.random() < 0.5:
            seq = seq.clone()
            seq[a:a + ln] = _reverse_strand(seq[a:a + ln])
        else:
            seg = seq[a:a + ln]
            rest = torch.cat([seq[:a], seq[a + ln:]])
            d = int(rng.integers(0, rest.numel() + 1))
            seq = torch.cat([rest[:d], seg, rest[d:]])
    return seq


def _plant_repeats(gen, rng: np.random.Generator, anc, share: float):
    """Copies of a 6 kbp and a 300 bp family written over anc at non-overlapping places."""
    torch = _torch()
    dev = anc.device
    L = anc.numel()
    unit = int(round(share * L / (20 * 300 + 6_000)))  # copies of the 6 kbp family
    tiles = L // 6_000
    if unit == 0 or tiles == 0:
        return anc
    unit = min(unit, tiles // 2)
    long_cons = _random_bases(gen, 6_000, 0.41, dev)
    short_cons = _random_bases(gen, 300, 0.41, dev)
    order = torch.randperm(tiles, generator=gen, device=dev)
    long_tiles, free = order[:unit], order[unit:]
    body = anc[:tiles * 6_000].view(tiles, 6_000)
    for s in range(0, unit, 1 << 14):
        idx = long_tiles[s:s + (1 << 14)]
        rates = 0.10 + 0.05 * torch.rand(idx.numel(), generator=gen, device=dev)
        body[idx] = _substitute_rows(gen, long_cons.repeat(idx.numel(), 1), rates)
    # the short copies go into 300 bp sub-tiles of the tiles left free
    sub = body.view(tiles * 20, 300)
    n_short = min(20 * unit, free.numel() * 20)
    cand = (free[:, None] * 20 + torch.arange(20, device=dev)[None, :]).reshape(-1)
    pick = cand[torch.randperm(cand.numel(), generator=gen, device=dev)[:n_short]]
    for s in range(0, n_short, 1 << 18):
        idx = pick[s:s + (1 << 18)]
        rates = 0.10 + 0.05 * torch.rand(idx.numel(), generator=gen, device=dev)
        sub[idx] = _substitute_rows(gen, short_cons.repeat(idx.numel(), 1), rates)
    return anc


def mammal_set(genome_len: int = 3_000_000_000, leaves: int = 8, seed: int = 1607,
               repeat_share: float = 0.45, device="cuda") -> List:
    """The leaves (uint8 CUDA tensors of about genome_len bases each)."""
    torch = _torch()
    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    anc = _random_bases(gen, genome_len, 0.41, dev)
    anc = _plant_repeats(gen, rng, anc, repeat_share)
    out: List = []

    def evolve(seq, n: int) -> None:
        if n == 1:
            out.append(seq.contiguous())
            return
        left = int(rng.integers(1, n))
        for part in (left, n - left):
            rate = float(rng.uniform(0.002, 0.012))  # per-edge divergence
            child = _substitute(gen, seq.clone(), rate * 10 / 11)
            child = _indels(gen, rng, child, rate / 11, 10)
            child = _structural(gen, rng, child, int(rng.integers(0, 3)), 1_000, 20_000)
            evolve(child, part)
            del child

    evolve(anc, leaves)
    return out


def concat_device(seqs) -> Tuple[object, np.ndarray]:
    """(one CUDA uint8 tensor of all bases, host offsets) of a list of CUDA tensors."""
    torch = _torch()
    lens = np.array([int(s.numel()) for s in seqs], dtype=np.uint64)
    off = np.zeros(len(seqs) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    return torch.cat(list(seqs)), off
