"""Choose the filter size b, bits per item h and round count for an input.

A larger Bloom filter leaves fewer false candidates for the exact second pass
(section "Theoretical Analysis and Comparison": the false-positive rate falls
with b / E); more rounds lower the peak memory -- one round's filter and
table -- at the cost of time (section "Multiple Rounds", Table 5). The paper
leaves the automatic choice of b and the number of rounds to future work
(Discussion). This tuner measures rather than models: it runs the library on
a sample of the input (the same-length prefix of every string) for each
candidate (b, h), with b scaled so that the filter has the same bits per base
as it would on the whole input, and keeps the fastest configuration whose
full-size workspace fits the memory budget, raising the round count only when
one round does not fit. A scaled-down filter can sit in L2 where the full one
does not, so the sample misranks filters of different sizes: the fastest
candidate of each filter size (up to ``refine`` sizes) is timed again on the
whole input before the choice. Last, the chosen configuration is timed on the
whole input with each launch shape of ``launch_shapes`` (resident blocks per
SM of the pass kernels; 0 = as many as fit) and keeps the fastest.

Every run goes through the C ABI (``twopaco.DeviceBuild``); nothing here
computes junctions.
"""
from __future__ import annotations

import math
import statistics
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import genomes, twopaco


@dataclass
class Trial:
    bits: int            # filter bits for the full input
    hashes: int
    rounds: int
    sample_ms: float     # mean time of one run on the sample
    est_full_ms: float   # sample time scaled to the full input
    workspace: int       # full-size workspace bytes
    candidates: float    # share of positions left after pass 1 (sample)
    table_slots: int = 0        # full-size table reserve the workspace was sized with
    candidate_records: int = 0  # full-size candidate list the workspace was sized with


@dataclass
class Choice:
    bits: int
    hashes: int
    rounds: int
    workspace: int
    est_full_ms: float
    trials: List[Trial] = field(default_factory=list)
    table_slots: int = 0
    candidate_records: int = 0
    blocks_per_sm: int = 0               # the chosen launch shape (0 = all that fit)
    shape_ms: Dict[int, float] = field(default_factory=dict)  # full-input ms per shape tried

    def options(self, **extra) -> twopaco.Options:
        """Options for the chosen configuration, with the table and list sizes its
        ``workspace`` was computed for (a table that still overflows is grown by the
        host builds and reported by the device runs) and its launch shape."""
        kw = dict(hashes=self.hashes, table_slots=self.table_slots,
                  candidate_records=self.candidate_records, launch_blocks_per_sm=self.blocks_per_sm)
        kw.update(extra)
        return twopaco.Options(**kw)


def prefix_sample(seqs: Sequence[np.ndarray], fraction: float, k: int) -> List[np.ndarray]:
    """The same-length prefix of every string, about ``fraction`` of all bases."""
    total = sum(int(s.size) for s in seqs)
    per = max(k + 1, int(math.ceil(total * fraction / max(1, len(seqs)))))
    return [np.ascontiguousarray(s[:per]) for s in seqs]


def full_workspace(total_bases: int, n_seqs: int, k: int, bits: int, rounds: int, hashes: int,
                   table_slots: int, candidate_records: int) -> int:
    opts = twopaco.Options(hashes=hashes, table_slots=table_slots,
                           candidate_records=candidate_records, partition_bins=65536)
    return twopaco.twopaco_workspace_size(total_bases, n_seqs, k, bits, rounds, opts)


def _pow2_at_least(x: float) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1.0, x)))))


def _time_run(run: twopaco.DeviceBuild, repeats: int) -> Tuple[float, Dict[str, int]]:
    import torch
    run.run()
    stats = run.stats()
    times = []
    for _ in range(repeats):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        run.run()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times), stats


def tune(seqs: Sequence[np.ndarray], k: int, budget_bytes: Optional[int] = None,
         bits_per_base: Sequence[float] = (4, 8, 16, 32), hashes: Sequence[int] = (3, 4, 6, 8),
         rounds: Sequence[int] = (1, 2, 4, 8, 16), sample_fraction: float = 0.1,
         repeats: int = 3, both_strands: bool = True, device: str = "cuda",
         refine: int = 4, launch_shapes: Sequence[int] = (0,)) -> Choice:
    """Measure candidate configurations on a sample; return the fastest that fits."""
    seqs = [np.ascontiguousarray(s, dtype=np.uint8) for s in seqs]
    total = sum(int(s.size) for s in seqs)
    sample = prefix_sample(seqs, sample_fraction, k)
    s_bases, s_off = genomes.concat(sample)
    scale = total / max(1, int(s_bases.size))
    trials: List[Trial] = []
    for r in sorted(rounds):
        fitting = []
        for bpb in bits_per_base:
            bits = max(256, _pow2_at_least(bpb * total))
            s_bits = max(256, _pow2_at_least(bpb * s_bases.size))
            for h in hashes:
                run = twopaco.DeviceBuild(s_bases, s_off, k, s_bits, r,
                                          twopaco.Options(hashes=h, both_strands=both_strands),
                                          device=device)
                ms, st = _time_run(run, repeats)
                # full-size table and candidate list from the sample's own sizes
                slots = _pow2_at_least(st["table_slots"] * scale * 1.25)
                cand_share = st["pass1_marks"] / max(1, st["positions"])
                # 8-byte list units hold two 32-bit records below 2^31 bases
                per_unit = 2 if total < (1 << 31) else 1
                recs = int(cand_share * total / r * 1.25 / per_unit) + (1 << 16)
                ws = full_workspace(total, len(seqs), k, bits, r, h, slots, recs)
                t = Trial(bits, h, r, ms, ms * scale, ws, cand_share, slots, recs)
                trials.append(t)
                if budget_bytes is None or ws <= budget_bytes:
                    fitting.append(t)
                del run
        if fitting:
            ranked = sorted(fitting, key=lambda t: (t.est_full_ms, t.workspace))
            if refine > 0 and len(ranked) > 1:
                # the sample's best (h, rounds) for every filter size, fastest sizes first
                per_size, seen = [], set()
                for t in ranked:
                    if t.bits not in seen:
                        seen.add(t.bits)
                        per_size.append(t)
                ranked = per_size[:refine]
                bases, off = genomes.concat(seqs)
                for t in ranked:  # the sample's estimate, replaced by a full-size time
                    run = twopaco.DeviceBuild(bases, off, k, t.bits, t.rounds,
                                              twopaco.Options(hashes=t.hashes,
                                                              both_strands=both_strands),
                                              device=device)
                    t.est_full_ms, _ = _time_run(run, max(1, repeats - 1))
                    del run
                ranked = sorted(ranked, key=lambda t: (t.est_full_ms, t.workspace))
            best = ranked[0]
            shape, shape_ms = 0, {}
            if len(launch_shapes) > 1:
                bases, off = genomes.concat(seqs)
                for bps in launch_shapes:
                    run = twopaco.DeviceBuild(bases, off, k, best.bits, best.rounds,
                                              twopaco.Options(hashes=best.hashes, both_strands=both_strands,
                                                              launch_blocks_per_sm=bps),
                                              device=device)
                    shape_ms[bps], _ = _time_run(run, max(1, repeats))
                    del run
                shape = min(shape_ms, key=lambda b: (shape_ms[b], b))
            return Choice(best.bits, best.hashes, best.rounds, best.workspace,
                          shape_ms.get(shape, best.est_full_ms), trials, best.table_slots,
                          best.candidate_records, shape, shape_ms)
    raise ValueError("no configuration fits the memory budget")
