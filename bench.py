#!/usr/bin/env python3
"""Throughput of two-pass junction detection (Gbp/s of genome input).

One step = one full build: pack, the class cut and class map (rounds > 1),
every round's two passes (Bloom-filter insert and probe, exact-table insert
and classify) and the emit of the sorted junction positions of every genome.

The headline workload is the mammal-scale configuration, the largest that
one GPU holds: 8 genomes of about 3 Gbp (24 Gbp) at the leaves of a seeded
random tree (45% repeats, 1-8% between leaves), drawn on the GPU, k = 25, a
2^36-bit filter with 4 hashes, 4 rounds (one round does not fit one GPU: its
candidate list, table and output would need more than its memory). ``value``
is measured with the ASCII resident in device memory; ``e2e`` streams it from
page-locked host memory through the library's streamed entry point and reads
the junction positions back, every step. The input (24 GB) is far larger than
L2, so nothing is flushed between steps.

Beside it the line carries the bacterial-size set (7 genomes of 4.6-5.6 Mbp,
2^28 bits, 1 round; L2 flushed between steps), the batched 62-genome set and
the served request stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload mammal_set|bacterial_set|plain_single] [--genome-len L]

Under torchrun the build is split by k-mer class (one process per GPU, rounds
r with r % N == rank, C_final merged by one all-reduce; at least N rounds):
``value`` is the one genome set's bases over the slowest rank's time
(strong scaling). ``--impl reference`` times the CPU oracle on a bounded
sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gbp/s genome input through both passes, k=25, 1 GB300; % roofline; p99 latency"
UNIT = "Gbp/s"
K = 25
FLUSH_BYTES = 512 << 20
CPU_SAMPLE_BASES = 100_000_000   # cpu_baseline leg: about 15 s of oracle work on 16 cores
REF_STEP_BASES = 4_000_000       # reference arm: one bounded sample per step (all host cores)
MAMMAL_GENOME_LEN = 3_000_000_000

WORKLOADS = {
    "mammal_set": {
        "filter_bits": 1 << 36, "hashes": 4, "rounds": 4,
        "desc": "mammal_set: 8 genomes of ~3 Gbp (24 Gbp) at the leaves of a seeded random binary tree "
                "(seed 1607, drawn on the GPU): 41% GC ancestor, 45% repeats (6 kbp and 300 bp families "
                "at 10-15% divergence), per-edge 0.2-1.2% SNPs and 1-10 bp indels at 10:1 plus 0-2 "
                "inversions/transpositions of 1-20 kbp"},
    "bacterial_set": {
        "filter_bits": 1 << 28, "hashes": 4, "rounds": 1,
        "desc": "bacterial_set: 7 related genomes of 4.6-5.6 Mbp (seed 1603; 50% GC ancestor, 1% SNPs, "
                "0.1% indels, 20 inversions/transpositions of 1-50 kbp, 1.5 kbp repeat x30)"},
    "plain_single": {
        "filter_bits": 1 << 24, "hashes": 3, "rounds": 1,
        "desc": "plain_single: 4 related 1 Mbp genomes (seed 1602; uniform ancestor, 0.5% SNPs, "
                "0.05% indels, 300 bp repeat x200 at 5%)"},
}


def workload_config(name: str, total_bases: int, rounds: int = None, world: int = 1) -> dict:
    w = WORKLOADS[name]
    big = total_bases > (256 << 20)
    return {
        "workload": w["desc"],
        "total_bases": int(total_bases),
        "k": K, "filter_bits": w["filter_bits"], "hashes": w["hashes"],
        "rounds": rounds or w["rounds"], "both_strands": True,
        "l2": (f"input ({total_bases / 1e9:.1f} GB) larger than L2: no flush" if big else
               f"flushed between timed steps ({FLUSH_BYTES >> 20} MiB write); input < L2"),
        "launch": "one CUDA-graph replay of the whole run per step (twopaco_plan_launch)" if world == 1
                  else "class-sharded: twopaco_shard_begin/rounds per rank, C_final all-reduced, "
                       "rank 0 writes the output",
    }


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="mammal_set", choices=sorted(WORKLOADS))
    p.add_argument("--genome-len", type=int, default=MAMMAL_GENOME_LEN,
                   help="mammal_set: bases per genome (a smaller slice of the same recipe)")
    p.add_argument("--rounds", type=int, default=0, help="override the workload's rounds")
    p.add_argument("--filter-bits", type=int, default=0,
                   help="override the workload's filter size (e.g. a slice at the same bits per base)")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--bacterial", type=int, default=1,
                   help="1: add the bacterial-size set's own line (when the headline is another workload)")
    p.add_argument("--batched", type=int, default=1,
                   help="1: add the batched leg (62 genomes in one tuned build vs one build per genome)")
    p.add_argument("--serve-requests", type=int, default=600,
                   help="requests of the served leg (Poisson, 20/s: 600 is 30 s); 0 skips it")
    return p.parse_args()


def sample_prefix(seqs, total):
    """A bounded sample: the same-length prefix of every genome, ~total bases."""
    per = max(1, total // len(seqs))
    return [s[:per] for s in seqs]


def oracle_gbps(seqs, k, threads: int = 1) -> float:
    """Throughput of the CPU oracle on seqs (with threads > 1: the partition-parallel
    form of the definition, each thread owning one hash class of the k-mers)."""
    import oracle
    from paper_1602_05856_gb300 import genomes
    bases, off = genomes.concat(seqs)
    t = time.perf_counter()
    oracle.junctions((bases, off), k, threads=threads)
    return bases.size / (time.perf_counter() - t) / 1e9


def note(msg: str) -> None:
    """Progress on stderr (stdout carries only the JSON line)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            if self.uuid and self.uuid not in f[1] and f[1] not in self.uuid:
                continue
            rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[6:10]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# Algorithmic work of every kernel over one step, from the run's own counters:
# (amount, kind) where kind names the roofline denominator: "rand_or" / "rand_read"
# are random 64-bit atomic ORs / 8-byte loads into the structure the kernel hits
# (one per unit), "hbm" streaming bytes.
def kernel_work(name, st, m, n_seqs, table_bytes, rounds=1):
    pos = st["positions"]
    cand = st["pass1_marks"]
    junc = st["pass2_marks"]
    # the region-ordered first pass: every round reads the class and region planes
    if name == "ord_scatter":  # planes + the members' k-mers; an 8 B record and a 2 B rank per member
        return rounds * (2 * m + m / 4) + 10 * pos, "hbm"
    if name == "ord_or":
        return pos, "l2_or"         # one OR per record into an L2-resident filter region
    if name == "ord_probe":
        return pos, "l2_read"       # one filter word load per record from an L2-resident region
    if name == "ord_classify":
        return cand, "l2_read"      # one table lookup per candidate record in an L2-resident region
    if name == "ord_gather":  # planes + ranks + decision bits; C_temp and the list written
        return rounds * (2 * m + m / 8) + 2 * pos + pos / 8 + 8 * cand, "hbm"
    if name == "pass1_insert":
        return pos, "rand_or"       # one random filter word OR per position
    if name == "pass1_probe":
        return pos, "rand_read"     # one random filter word load per position
    if name == "pass2_insert":
        return cand, "rand_or"      # one table slot (CAS / OR) per candidate
    if name == "pass2_classify":
        return cand, "rand_read"    # one table slot load per candidate
    if name == "partition_count":
        return pos, "rand_read"     # one random filter word test per position
    if name == "pack":
        return m + m / 4, "hbm"     # ASCII read + packed write (bytes)
    if name == "class_map":
        return m / 4 + m, "hbm"     # packed read + one class byte written per position
    if name == "table_clear":
        return table_bytes, "hbm"
    if name == "emit":
        return m / 8 + 8 * junc, "hbm"  # C_final read + positions written (bytes)
    return None, None


def kernel_code_digest() -> str:
    """sha256 of csrc/twopaco_kernels.cu without comments, blank lines and edge whitespace."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_1602_05856_gb300", "csrc", "twopaco_kernels.cu")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = [re.sub(r"//.*$", "", l).strip() for l in src.splitlines()]
    return hashlib.sha256("\n".join(l for l in lines if l).encode()).hexdigest()


def ncu_traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` on `workload`, from a committed ncu summary.

    profiles/dram_traffic_*.md carry lines ``dram-traffic <workload> <kernel> <bytes>
    sha256:<digest of the code of csrc/twopaco_kernels.cu when captured>`` (the digest
    of the source with its comments and blank lines removed, see kernel_code_digest); a
    figure taken from older kernel code does not count (None).
    """
    import glob
    import re
    digest = kernel_code_digest()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "dram_traffic_*.md"))):
        for line in open(path):
            m = re.match(r"dram-traffic (\S+) (\S+) (\d+) sha256:([0-9a-f]{64})\s*$", line.strip())
            if m and m.group(1) == workload and m.group(2) == kernel and m.group(4) == digest:
                return int(m.group(3))
    return None


# ---------------------------------------------------------------------------
# inputs and sizes
# ---------------------------------------------------------------------------

def load_workload(name, genome_len, dev):
    """(device bases, host offsets, host sequence views or None) of a workload."""
    import torch
    if name == "mammal_set":
        from paper_1602_05856_gb300 import genomes_gpu as GG
        leaves = GG.mammal_set(genome_len=genome_len, device=dev)
        d_bases, off = GG.concat_device(leaves)
        del leaves
        torch.cuda.empty_cache()
        return d_bases, off, None
    from paper_1602_05856_gb300 import genomes
    seqs = genomes.named_set(name)
    bases, off = genomes.concat(seqs)
    return torch.from_numpy(bases).to(dev), off, seqs


def sized_options(T, name, m, rounds, stream=0):
    """Options and output capacity: the defaults for inputs that fit them; for the
    mammal-scale set a pass-2 table, candidate list and output sized from its measured
    shares (28% of the positions survive pass 1 at 4 rounds, 26.6% are junctions, about
    3% of a round's positions are distinct candidates, which a table of 2.5 times as
    many slots takes) with room to spare -- a run that still overflows fails loudly."""
    w = WORKLOADS[name]
    if name != "mammal_set":
        return T.Options(hashes=w["hashes"], cuda_stream=stream), None
    per_round = m // rounds
    slots = 1 << max(20, int(np.ceil(np.log2(max(per_round * 0.15, 1)))))
    return (T.Options(hashes=w["hashes"], table_slots=slots, candidate_records=per_round // 2,
                      cuda_stream=stream), int(m * 0.285))


def l2_or_hbm_peaks(build, filter_bytes):
    """Random-access rates (accesses/s) of this GPU on a buffer of the filter's size:
    64-bit atomic ORs and 8-byte loads, each the better of two address generators
    (a 64-bit mixer per access, or a 32-bit linear congruential sequence)."""
    import ctypes
    peaks = ctypes.CDLL(build.build_peaks())
    peaks.peaks_l2_random_rate.restype = ctypes.c_double
    peaks.peaks_l2_random_rate.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
    buf = max(1 << 20, min(int(filter_bytes), 8 << 30))
    r = {"or_mix": peaks.peaks_l2_random_rate(1, buf, 64, 5),
         "or_lcg": peaks.peaks_l2_random_rate(4, buf, 1024, 5),
         "read_mix": peaks.peaks_l2_random_rate(2, buf, 64, 5),
         "read_lcg": peaks.peaks_l2_random_rate(5, buf, 1024, 5),
         "sector_read_lcg": peaks.peaks_l2_random_rate(3, buf, 1024, 5),
         "buffer_bytes": buf}
    r["or"] = max(r["or_mix"], r["or_lcg"])
    r["read"] = max(r["read_mix"], r["read_lcg"])
    # and on one filter region of the region-ordered first pass (32 MiB, in L2)
    reg = min(int(filter_bytes), 32 << 20)
    r["l2_or"] = max(peaks.peaks_l2_random_rate(1, reg, 64, 5), peaks.peaks_l2_random_rate(4, reg, 1024, 5))
    r["l2_read"] = max(peaks.peaks_l2_random_rate(2, reg, 64, 5), peaks.peaks_l2_random_rate(5, reg, 1024, 5))
    r["l2_bytes"] = reg
    return r


def roofline(prof, st, m, n, table_bytes, peaks, hbm_peak, peaks_json, workload, in_l2, steps, rounds=1):
    """The roofline object of the dominant modelled kernel; prof sums `steps` steps."""
    modelled = [kv for kv in prof.items() if kernel_work(kv[0], st, m, n, table_bytes, rounds)[0] is not None]
    name, rec = max(modelled or prof.items(), key=lambda kv: kv[1]["ms"])
    ms = rec["ms"] / rec["launches"]
    amount, kind = kernel_work(name, st, m, n, table_bytes, rounds)
    amount = (amount or 0.0) * steps / rec["launches"]  # a step's work shared over its launches
    if kind in ("l2_or", "l2_read"):
        pk = peaks[kind] / 1e9
        achieved = amount / (ms * 1e-3) / 1e9
        roof = {"bound": "l2", "achieved": achieved, "peak": pk, "unit": "Gaccess/s", "frac": achieved / pk,
                "peak_source": "measured in this run: random " + ("8-byte loads" if kind == "l2_read" else
                               "64-bit atomic ORs") + f" over a {peaks['l2_bytes'] >> 20} MiB buffer (one filter "
                               "region, in L2), all SMs, the better of two address streams, best of 5 (of measured)"}
    elif kind in (None, "hbm"):
        achieved = amount / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks_json
                               else "fallback 6.8 TB/s (of fallback)"}
    else:
        pk = (peaks["read"] if kind == "rand_read" else peaks["or"]) / 1e9
        achieved = amount / (ms * 1e-3) / 1e9
        where = "L2-resident" if in_l2 else "in HBM, beyond L2"
        roof = {"bound": "l2" if in_l2 else "hbm_random", "achieved": achieved, "peak": pk,
                "unit": "Gaccess/s", "frac": achieved / pk if pk > 0 else None,
                "peak_source": f"measured in this run: random "
                               + ("8-byte loads" if kind == "rand_read" else "64-bit atomic ORs")
                               + f" over a {peaks['buffer_bytes'] >> 20} MiB buffer ({where}, the "
                               "filter's size), all SMs, the better of a 64-bit-mixer and a "
                               "32-bit-LCG address stream, best of 5 (of measured)"}
    roof["kernel"] = name
    roof["traffic"] = ncu_traffic(workload, name)
    roof["traffic_unit"] = "DRAM bytes per launch (ncu, cold cache)"
    roof["kernel_ms"] = ms
    return roof


# ---------------------------------------------------------------------------
# device-resident timing
# ---------------------------------------------------------------------------

def time_steps(T, step, stream, steps, warmup, flush, dev, graph):
    """Run warmup untimed steps, then time `steps` with CUDA events on `stream`.
    graph: every step replays a graph captured with profiling on, whose kernel events
    every replay records again (else the step's launches record new events)."""
    import torch
    for _ in range(max(warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    prof: dict = {}
    if not graph:
        T.twopaco_profile_enable(True)
    launches0 = T.twopaco_kernel_launches()
    wall0 = time.perf_counter()
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
        ends[i].synchronize()  # between steps: this step's kernel events are final
        for name, rec in T.twopaco_profile_kernels().items():
            p = prof.setdefault(name, {"launches": 0, "ms": 0.0})
            p["launches"] += rec["launches"]
            p["ms"] += rec["ms"]
        if not graph:
            T.twopaco_profile_enable(True)  # drop this step's records
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    launches = T.twopaco_kernel_launches() - launches0
    T.twopaco_profile_enable(False)
    return [s.elapsed_time(e) for s, e in zip(starts, ends)], prof, launches, wall


def kernels_summary(prof, steps):
    tot = sum(x["ms"] for x in prof.values()) or 1.0
    return {k: {"launches": v["launches"], "launches_per_step": v["launches"] / max(steps, 1),
                "ms_per_launch": v["ms"] / v["launches"], "ms_per_step": v["ms"] / max(steps, 1),
                "share": v["ms"] / tot} for k, v in prof.items()}


def device_leg(T, build, name, genome_len, rounds, args, world, rank, local, dist):
    """Device-resident throughput of one workload (and its e2e), as one dict."""
    import torch
    from paper_1602_05856_gb300 import shard
    dev = torch.device("cuda", local)
    w = WORKLOADS[name]
    rounds = rounds or w["rounds"]
    if world > 1:
        rounds = max(rounds, world)  # every rank owns at least one class
    # the random-access rates first, while the device holds nothing else
    peaks = l2_or_hbm_peaks(build, w["filter_bits"] // 8)
    d_bases, off, seqs = load_workload(name, genome_len, dev)
    m, n = int(off[-1]), len(off) - 1
    stream = torch.cuda.current_stream(dev)
    opts, capacity = sized_options(T, name, m, rounds)
    run = T.DeviceBuild(d_bases, off, K, w["filter_bits"], rounds, opts, device=f"cuda:{local}",
                        capacity=capacity)
    in_l2 = w["filter_bits"] // 8 <= (64 << 20)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev) if m <= (256 << 20) else None
    if world == 1:
        T.twopaco_profile_enable(True)  # before the capture: replays record the captured events
        run.capture()  # the whole run as one CUDA graph

        def step():
            run.run(stream)
    else:
        def step():
            shard.sharded_build(run, rank, world, dist)
    props = torch.cuda.get_device_properties(dev)
    sampler = ClockSampler(str(getattr(props, "uuid", "") or ""))
    barrier(world)
    sampler.start()
    step_ms, prof, launches, wall = time_steps(T, step, stream, args.steps, args.warmup, flush, dev,
                                               graph=world == 1)
    barrier(world)
    clocks = sampler.stop()
    run.release_plan()
    st = run.stats(stream)  # raises on any recorded failure (overflow, bad base, timeout)
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ms, world)
    junctions = int(run.out_offsets[-1].item()) if rank == 0 else st["pass2_marks"]
    table_bytes = st["table_slots"] * (8 if K <= 27 else 16 if K <= 31 else 32)
    peaks_json = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks_json.get("hbm_gbs", 6800.0))
    out = {"name": name, "m": m, "n": n, "rounds": rounds, "ms": ms_max, "step_ms": step_ms,
           "value": m / (ms_max * 1e-3) / 1e9, "launches": launches, "clocks": clocks, "wall": wall,
           "stats": {k: st[k] for k in ("positions", "pass1_marks", "pass2_marks", "table_slots", "ordered_rounds")}
                    | {"junctions": junctions},
           "kernels": kernels_summary(prof, args.steps),
           "roofline": roofline(prof, st, m, n, table_bytes, peaks, hbm_peak, peaks_json, name, in_l2,
                                args.steps, rounds),
           "random_access_peaks_g_per_s": {k: (v / 1e9 if k not in ("buffer_bytes", "l2_bytes") else v)
                                           for k, v in peaks.items()}}
    out["e2e"] = e2e_leg(T, run, d_bases, off, seqs, name, opts, rounds, args, world, rank, dev,
                         junctions) if args.e2e_steps > 0 else None
    out["cpu_sample"] = cpu_sample(d_bases, off, seqs) if rank == 0 and not args.no_cpu_baseline else None
    del run, d_bases
    torch.cuda.empty_cache()
    if hasattr(torch._C, "_host_emptyCache"):
        torch._C._host_emptyCache()  # the page-locked e2e buffers (tens of GB at full size)
    return out


def e2e_leg(T, run, d_bases, off, seqs, name, opts, rounds, args, world, rank, dev, junctions):
    """The same metric through the public API with host buffers, copies inside the timed
    region: the mammal set streamed from page-locked host memory through
    twopaco_run_streamed and the junction positions read back; the smaller sets through
    twopaco_build_ctx on a reused context."""
    import torch
    m, n = int(off[-1]), len(off) - 1
    w = WORKLOADS[name]
    times = []
    if name == "mammal_set" or world > 1:
        host = torch.empty(m, dtype=torch.uint8, pin_memory=True)
        host.copy_(d_bases)
        staging = torch.empty(1 << 29, dtype=torch.uint8, device=dev)  # two 256 MiB halves
        out_pos = torch.empty(max(junctions, 1), dtype=torch.int64, pin_memory=True)
        out_off = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
        stream = torch.cuda.current_stream(dev)
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            if world == 1:
                run.run_streamed(host, staging, stream)
            else:  # every rank copies its own input in, then the class-sharded rounds
                from paper_1602_05856_gb300 import shard
                run.bases.copy_(host, non_blocking=True)
                shard.sharded_build(run, rank, world, torch.distributed)
            if rank == 0:  # the rank that wrote the output reads it back
                out_off.copy_(run.out_offsets, non_blocking=True)
                stream.synchronize()
                total = int(out_off[-1].item())
                if total != junctions:
                    raise RuntimeError("the streamed run and the device run disagree")
                out_pos[:total].copy_(run.out_positions[:total], non_blocking=True)
            stream.synchronize()
            if i:
                times.append(time.perf_counter() - t0)
        api = ("twopaco_run_streamed: page-locked host ASCII streamed through two 256 MiB staging "
               "halves (copies overlapped with the packing), run, D2H of offsets and positions into "
               "page-locked memory")
        h2d = m
    else:
        pinned = torch.empty(m, dtype=torch.uint8, pin_memory=True)
        pinned.copy_(d_bases)
        host = pinned.numpy()
        host_seqs = [host[int(off[t]):int(off[t + 1])] for t in range(n)]
        ctx = T.Context()
        for i in range(args.e2e_steps + 1):
            t0 = time.perf_counter()
            got, _ = ctx.build(host_seqs, K, w["filter_bits"], rounds, T.Options(hashes=w["hashes"]),
                               copy=False)
            if i:
                times.append(time.perf_counter() - t0)
            if sum(g.size for g in got) != junctions:
                raise RuntimeError("host API and device run disagree")
        ctx.close()
        api = ("twopaco_build_ctx: pinned host ASCII in, H2D, run, D2H of offsets and positions into "
               "pinned memory, on a reused context")
        h2d = m + 8 * (n + 1)
    sec = max_over_ranks(statistics.mean(times), world)
    return {"value": m / sec / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": 8 * (n + 1) + 8 * junctions, "api": api, "ms_per_step": sec * 1e3}


def cpu_sample(d_bases, off, seqs):
    """Prefixes of every genome, ~CPU_SAMPLE_BASES in all, as host arrays."""
    n = len(off) - 1
    per = max(1, CPU_SAMPLE_BASES // n)
    out = []
    for t in range(n):
        a = int(off[t])
        ln = min(per, int(off[t + 1]) - a)
        out.append(d_bases[a:a + ln].cpu().numpy() if seqs is None else seqs[t][:ln])
    return out


# ---------------------------------------------------------------------------
# batched and served legs
# ---------------------------------------------------------------------------

def batched_leg(T, genomes, dev):
    """The 62-genome set (310 Mbp) as one build: with the autotuner's (b, h) in one launch per
    loop replayed as a CUDA graph (the batched path), against the same build issued the way a
    per-genome loop issues it -- every loop launched once per genome, without graph capture --
    and against an untuned filter. All three compute the same graph; their outputs are
    compared here. One build per genome (62 separate, smaller graphs) is reported beside them
    as context."""
    import torch
    from paper_1602_05856_gb300 import autotune
    seqs = genomes.named_set("batched_set")
    bases, off = genomes.concat(seqs)
    m = int(off[-1])
    choice = autotune.tune(seqs, K, budget_bytes=120 << 30, bits_per_base=(2, 4, 8, 16),
                           hashes=(3, 4, 6), rounds=(1,), sample_fraction=0.1, repeats=2,
                           launch_shapes=(0, 2, 4))
    bpb = choice.bits / m
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        a = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        b = [torch.cuda.Event(enable_timing=True) for _ in range(reps)]
        for i in range(reps):
            a[i].record(stream)
            fn()
            b[i].record(stream)
        torch.cuda.synchronize()
        return statistics.mean(x.elapsed_time(y) for x, y in zip(a, b))

    def joint(bits, hashes, per_string=False, shape=0):
        run = T.DeviceBuild(bases, off, K, bits, 1,
                            T.Options(hashes=hashes, per_string_launches=per_string,
                                      launch_blocks_per_sm=shape), device=dev)
        if not per_string:
            run.capture()
        n0 = T.twopaco_kernel_launches()
        ms = timed(run.run, 5)
        launches = (T.twopaco_kernel_launches() - n0) // 6
        st = run.stats()
        res = run.result()
        run.release_plan()
        return ms, st, res, launches

    batched_ms, st, want, batched_launches = joint(choice.bits, choice.hashes, shape=choice.blocks_per_sm)
    per_ms, _, got, per_launches = joint(choice.bits, choice.hashes, per_string=True)
    plain_ms, _, got_plain, _ = joint(1 << 30, 4)  # the paper's filter size at this scale, 4 hashes
    same = all(np.array_equal(a, b) for a, b in zip(want, got)) and \
        all(np.array_equal(a, b) for a, b in zip(want, got_plain))
    if not same:
        raise RuntimeError("the batched, per-genome and untuned launches disagree")
    # context: one separate build per genome through twopaco_run_device, on one workspace
    d_bases = torch.from_numpy(bases).to(dev)
    lens = [int(off[t + 1] - off[t]) for t in range(len(seqs))]
    bits_of = [1 << max(8, int(np.ceil(np.log2(max(bpb * ln, 1.0))))) for ln in lens]
    opts = T.Options(hashes=choice.hashes, cuda_stream=int(stream.cuda_stream))
    ws_bytes = max(T.twopaco_workspace_size(ln, 1, K, bt, 1, opts) for ln, bt in zip(lens, bits_of))
    ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=dev)
    ws_ptr = (ws.data_ptr() + 255) // 256 * 256
    offs = torch.zeros((len(seqs), 2), dtype=torch.int64, device=dev)
    offs[:, 1] = torch.tensor(lens, dtype=torch.int64)
    out_off = torch.zeros(2, dtype=torch.int64, device=dev)
    out_pos = torch.empty(max(lens), dtype=torch.int64, device=dev)

    def per_genome():
        for t, (ln, bt) in enumerate(zip(lens, bits_of)):
            T.twopaco_run_device(d_bases.data_ptr() + int(off[t]), offs[t].data_ptr(), 1, ln, K, bt, 1,
                                 opts, ws_ptr, ws_bytes, out_off.data_ptr(), out_pos.data_ptr(),
                                 int(out_pos.numel()))

    single_ms = timed(per_genome, 3)
    return {"genomes": len(seqs), "bases": m, "k": K,
            "tuned": {"filter_bits": choice.bits, "hashes": choice.hashes, "rounds": choice.rounds,
                      "trials": len(choice.trials), "launch_blocks_per_sm": choice.blocks_per_sm,
                      "launch_shape_ms": {str(k): v for k, v in choice.shape_ms.items()}},
            "batched_gbps": m / (batched_ms * 1e-3) / 1e9, "batched_ms": batched_ms,
            "batched_launches_per_build": batched_launches,
            "per_genome_launches_gbps": m / (per_ms * 1e-3) / 1e9, "per_genome_launches_ms": per_ms,
            "per_genome_launches_per_build": per_launches,
            "untuned_gbps": m / (plain_ms * 1e-3) / 1e9, "untuned": {"filter_bits": 1 << 30, "hashes": 4},
            "same_output": same,
            "separate_builds_gbps": m / (single_ms * 1e-3) / 1e9, "separate_builds_ms": single_ms,
            "pass1_survivors": st["pass1_marks"] / max(1, st["positions"]),
            "note": "batched: one joint build (one launch per loop, graph replay) with the tuned "
                    "(b, h); per-genome launches: the same build with every loop launched once per "
                    "genome, no graph (identical output, checked); untuned: b = 2^30, h = 4 "
                    "(identical output, checked); separate builds: each genome built alone (62 "
                    "smaller graphs), context only"}


def served_leg(args, local):
    """The served configuration: a Poisson stream (20/s) of requests of 2-50 genome windows
    of 0.1-50 Mbp (log-uniform, from the bacterial recipe at 10x length), k 25/31, admitted
    by device memory under 120 GB into 4 slots whose work overlaps on the GPU; against every
    request run alone on an idle GPU."""
    from paper_1602_05856_gb300 import serve
    pool = serve.served_pool(lock=True)  # the server's resident, page-locked genome store

    def trace():
        return serve.served_requests(pool, args.serve_requests, serve.SERVED_RATE, seed=1606,
                                     genomes_range=serve.SERVED_GENOMES, mbp_range=serve.SERVED_MBP,
                                     digest_only=True)

    reqs = trace()
    slots = [serve.GpuSlot(device=f"cuda:{local}") for _ in range(4)]
    for sl in slots:  # staging grown and the largest request run once: later requests hit the caches
        sl.reserve(reqs)
    import gc
    gc.collect()
    gc.disable()  # no collector pause inside the timed loops
    try:
        mix_rep = serve.Scheduler(slots, serve.SERVED_BUDGET).run(reqs)
        alone_rep = serve.run_alone(slots[0], trace())
    finally:
        gc.enable()
    same = all(x.digest == y.digest and x.digest is not None
               for x, y in zip(sorted(mix_rep.requests, key=lambda r: r.rid),
                               sorted(alone_rep.requests, key=lambda r: r.rid)))
    if not same:
        raise RuntimeError("a served request's junctions differ alone and in the mix")
    mix, alone = mix_rep.summary(), alone_rep.summary()
    bases = sum(r.bases for r in reqs)
    keys = ("p50_ms", "p95_ms", "p99_ms", "max_ms", "mean_ms", "throughput_gbps", "wall_s")
    return {"requests": args.serve_requests, "rate_per_s": serve.SERVED_RATE, "slots": 4,
            "budget_gb": serve.SERVED_BUDGET >> 30, "duration_s": reqs[-1].arrival,
            "offered_gbps": bases / reqs[-1].arrival / 1e9,
            "mix": {k: mix[k] for k in keys}, "alone": {k: alone[k] for k in keys},
            "same_results_alone_and_in_mix": same,
            "request_bases_mbp": {"mean": bases / len(reqs) / 1e6,
                                  "max": max(r.bases for r in reqs) / 1e6},
            "request_recipe": "2-50 windows of the 7 genomes of the bacterial recipe at 10x length "
                              "(46-56 Mbp, a page-locked resident store the windows copy from), window "
                              "lengths log-uniform 0.1-50 Mbp at uniform offsets, "
                              "k 25/31 alternating, ~8 filter bits per base, 4 hashes, pass-2 table "
                              "reserve half a slot per base (grown on overflow)"}


# ---------------------------------------------------------------------------
# the two arms
# ---------------------------------------------------------------------------

def run_ours(args, world, rank, local):
    import torch
    from paper_1602_05856_gb300 import build, genomes, twopaco as T

    torch.cuda.set_device(local)
    if rank == 0:  # one rank compiles (if anything is out of date); the others wait for it
        build.build()
    barrier(world)
    build.build()  # up to date now: only checks
    dist = None
    if world > 1:
        import torch.distributed as dist
    name = args.workload
    if args.filter_bits:
        WORKLOADS[name] = dict(WORKLOADS[name], filter_bits=int(args.filter_bits))
    note(f"{name}: device leg")
    head = device_leg(T, build, name, args.genome_len, args.rounds, args, world, rank, local, dist)
    note(f"{name}: {head['value']:.2f} Gbp/s")

    extra = {}
    if rank == 0 and world == 1 and args.bacterial and name != "bacterial_set":
        b = device_leg(T, build, "bacterial_set", 0, 0, args, 1, 0, local, None)
        extra["bacterial_set"] = {
            "value": b["value"], "unit": UNIT, "ms_per_step": b["ms"], "config":
                workload_config("bacterial_set", b["m"]), "roofline": b["roofline"],
            "e2e": b["e2e"], "stats": b["stats"], "kernels": b["kernels"], "gpu_launches": b["launches"],
            "random_access_peaks_g_per_s": b["random_access_peaks_g_per_s"], "clocks": b["clocks"]}
    if rank == 0 and world == 1 and args.batched:
        note("batched leg")
        extra["batched"] = batched_leg(T, genomes, torch.device("cuda", local))
    if rank == 0 and world == 1 and args.serve_requests > 0:
        note("served leg")
        extra["served"] = served_leg(args, local)

    cpu = None
    if rank == 0 and head["cpu_sample"] is not None:
        note("cpu baseline")
        sample = head["cpu_sample"]
        cores = host_cores()
        cpu = {"value": oracle_gbps(sample, K, threads=cores), "unit": UNIT, "cores": cores,
               "kind": "oracle",
               "sample": f"{sum(s.size for s in sample)} bases: the first {sample[0].size} bases of "
                         f"each of the {len(sample)} genomes of the timed input; the definition split "
                         f"over {cores} threads by k-mer hash class"}
    lat = sorted(head["step_ms"])
    out = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True,
        "scaling": "weak" if world == 1 else "strong", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": workload_config(name, head["m"], head["rounds"], world)
                  | {"parallelism": "single" if world == 1 else f"classes{world}"},
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "e2e": head["e2e"],
        "gpu_launches": head["launches"],
        "roofline": head["roofline"],
        "cpu_baseline": cpu,
        "clocks": head["clocks"],
        "stats": head["stats"],
        "kernels": head["kernels"],
        "random_access_peaks_g_per_s": head["random_access_peaks_g_per_s"],
        "timed_wall_s": head["wall"],
    } | extra
    if rank == 0:
        print(json.dumps(out), flush=True)


def reference_sample(name):
    """One bounded sample of the workload for the reference arm (host arrays)."""
    if name == "mammal_set":
        from paper_1602_05856_gb300 import genomes_gpu as GG
        leaves = GG.mammal_set(genome_len=REF_STEP_BASES // 8, device="cpu")
        return [x.numpy() for x in leaves], ("8 leaves of the mammal-scale recipe drawn at "
                                             f"{REF_STEP_BASES // 8} bases each")
    from paper_1602_05856_gb300 import genomes
    seqs = genomes.named_set(name)
    sample = sample_prefix(seqs, REF_STEP_BASES)
    return sample, f"the first {sample[0].size} bases of each of the {len(seqs)} genomes"


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_1602_05856_gb300 import genomes
    import oracle
    name = args.workload
    sample, what = reference_sample(name)
    sb, so = genomes.concat(sample)
    cores = host_cores()
    for _ in range(max(args.warmup, 0)):
        oracle.junctions((sb, so), K, threads=cores)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.junctions((sb, so), K, threads=cores)
        ts.append(time.perf_counter() - t)
    sec = statistics.mean(ts)
    value = sb.size / sec / 1e9
    full = 8 * args.genome_len if name == "mammal_set" else sum(s.size for s in genomes.named_set(name))
    desc = (f"{sb.size} bases per step: {what}; CPU oracle (plain definition) split over {cores} "
            f"threads by k-mer hash class")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": workload_config(name, full, args.rounds or None) | {"parallelism": "single"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
