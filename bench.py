#!/usr/bin/env python3
"""Throughput of two-pass junction detection (Gbp/s of genome input).

One step = one full build over the bacterial-size genome set (7 related
genomes of 4.6-5.6 Mbp, k = 25, a 2^28-bit filter with 4 hashes, 1 round):
pack, pass 1 (filter insert + probe), pass 2 (exact table insert +
classify) and the emit of sorted junction positions, all from ASCII already
resident in device memory. The input (35 MB) is smaller than L2, so a
512 MiB buffer is written between timed steps to flush it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank runs an independent replica of the workload on
its own GPU (the build of one genome set does not shard); ``value`` is the
bases of all replicas over the slowest rank's time. ``--impl reference``
times the CPU oracle on a bounded sample of the same workload instead.
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
WORKLOAD = "bacterial_set"
K = 25
FILTER_BITS = 1 << 28
HASHES = 4
ROUNDS = 1
FLUSH_BYTES = 512 << 20
CPU_SAMPLE_BASES = 8_000_000     # cpu_baseline leg: about 10 s of oracle work
REF_STEP_BASES = 4_000_000   # reference arm: one bounded sample per step (all host cores)


def workload_config(total_bases: int) -> dict:
    desc = ("bacterial_set: 7 related genomes of 4.6-5.6 Mbp (seed 1603; 50% GC ancestor, "
            "1% SNPs, 0.1% indels, 20 inversions/transpositions of 1-50 kbp, 1.5 kbp repeat x30)")
    if WORKLOAD == "plain_single":
        desc = ("plain_single: 4 related 1 Mbp genomes (seed 1602; uniform ancestor, 0.5% SNPs, "
                "0.05% indels, 300 bp repeat x200 at 5%)")
    return {
        "workload": desc,
        "total_bases": int(total_bases),
        "k": K, "filter_bits": FILTER_BITS, "hashes": HASHES, "rounds": ROUNDS,
        "both_strands": True,
        "l2": f"flushed between timed steps ({FLUSH_BYTES >> 20} MiB write); input 35 MB < L2",
        "launch": "one CUDA-graph replay of the whole run per step (twopaco_plan_launch)",
    }


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batched", type=int, default=1,
                   help="1: add the batched leg (62 genomes in one tuned build vs one build per genome)")
    p.add_argument("--serve-requests", type=int, default=100,
                   help="requests of the served leg (Poisson, 20/s); 0 skips it")
    p.add_argument("--workload", default=WORKLOAD, choices=["bacterial_set", "plain_single"],
                   help="plain_single: the 4 x 1 Mbp set (k=25, 2^24 bits, 3 hashes) for small captures")
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


# Algorithmic work of every kernel per launch, from the run's own counters:
# (unit, amount, kind) where kind names the roofline denominator.
def kernel_work(name, st, m, n_seqs, table_bytes):
    pos = st["positions"]
    cand = st["pass1_marks"]
    junc = st["pass2_marks"]
    if name == "pass1_insert":
        return pos, "l2_or"        # one random filter sector (read + ORs) per position
    if name == "pass1_probe":
        return pos, "l2_read"      # one random filter sector read per position
    if name == "pass2_insert":
        return cand, "l2_or"       # one table slot (CAS + OR) per candidate
    if name == "pass2_classify":
        return cand, "l2_read"     # one table slot read per candidate
    if name == "pack":
        return m + m / 4, "hbm"    # ASCII read + packed write (bytes)
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


def batched_leg(T, genomes, dev):
    """The 62-genome set (310 Mbp) as one build with the autotuner's (b, h), against the
    same genomes built one at a time (the single-instance path) at the same filter bits per
    base, both device-resident and timed with CUDA events. The two compute different graphs
    (one joint graph vs 62 separate ones): this compares throughput, not output."""
    import torch
    from paper_1602_05856_gb300 import autotune
    seqs = genomes.named_set("batched_set")
    bases, off = genomes.concat(seqs)
    m = int(off[-1])
    choice = autotune.tune(seqs, K, budget_bytes=120 << 30, bits_per_base=(2, 4, 8, 16),
                           hashes=(3, 4, 6), rounds=(1,), sample_fraction=0.1, repeats=2)
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

    def joint(bits, hashes):
        run = T.DeviceBuild(bases, off, K, bits, 1, T.Options(hashes=hashes), device=dev)
        run.capture()
        ms = timed(run.run, 5)
        st = run.stats()
        run.release_plan()
        return ms, st

    batched_ms, st = joint(choice.bits, choice.hashes)
    plain_ms, _ = joint(1 << 30, 4)  # the paper's filter size for inputs of this scale, 4 hashes
    # one genome at a time through twopaco_run_device, on one workspace and one output buffer
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
                      "trials": len(choice.trials)},
            "batched_gbps": m / (batched_ms * 1e-3) / 1e9, "batched_ms": batched_ms,
            "untuned_gbps": m / (plain_ms * 1e-3) / 1e9, "untuned": {"filter_bits": 1 << 30, "hashes": 4},
            "single_instance_gbps": m / (single_ms * 1e-3) / 1e9, "single_instance_ms": single_ms,
            "pass1_survivors": st["pass1_marks"] / max(1, st["positions"]),
            "note": "batched: one joint build of all genomes (one launch per kernel, graph replay) "
                    "with the tuned (b, h), and untuned with b = 2^30, h = 4; single instance: each "
                    "genome built alone, back to back (62 separate, far less branched graphs, so "
                    "throughput only)"}


def run_ours(args, world, rank, local):
    import torch
    from paper_1602_05856_gb300 import build, genomes, twopaco as T

    global WORKLOAD, FILTER_BITS, HASHES
    if args.workload == "plain_single":
        WORKLOAD, FILTER_BITS, HASHES = "plain_single", 1 << 24, 3

    torch.cuda.set_device(local)
    if rank == 0:  # one rank compiles (if anything is out of date); the others wait for it
        build.build()
    barrier(world)
    build.build()  # up to date now: only checks
    dev = torch.device("cuda", local)
    seqs = genomes.named_set(WORKLOAD)
    bases, off = genomes.concat(seqs)
    m, n = int(off[-1]), len(seqs)
    opts = T.Options(hashes=HASHES)
    run = T.DeviceBuild(bases, off, K, FILTER_BITS, ROUNDS, opts, device=f"cuda:{local}")
    stream = torch.cuda.current_stream(dev)

    # roofline denominators measured on this GPU: random 32-byte sectors of a
    # buffer the size of the filter
    import ctypes
    peaks = ctypes.CDLL(build.build_peaks())
    peaks.peaks_l2_random_rate.restype = ctypes.c_double
    peaks.peaks_l2_random_rate.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_int]
    l2_read = peaks.peaks_l2_random_rate(2, FILTER_BITS // 8, 64, 5)   # random 8-byte loads
    l2_or = peaks.peaks_l2_random_rate(1, FILTER_BITS // 8, 64, 5)     # random 64-bit ORs
    l2_sector = peaks.peaks_l2_random_rate(0, FILTER_BITS // 8, 64, 5)  # random 32-byte sectors

    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # the whole run is captured once as a CUDA graph (with its per-kernel events)
    T.twopaco_profile_enable(True)
    run.capture()
    for _ in range(max(args.warmup, 0)):
        run.run(stream)
    st = run.stats(stream)  # raises on any recorded failure
    torch.cuda.synchronize(dev)

    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    sampler = ClockSampler(uuid)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    prof: dict = {}
    barrier(world)
    torch.cuda.synchronize(dev)
    sampler.start()
    launches0 = T.twopaco_kernel_launches()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        run.run(stream)
        ends[i].record(stream)
        ends[i].synchronize()  # between steps: this replay's kernel events are final
        for name, rec in T.twopaco_profile_kernels().items():
            p = prof.setdefault(name, {"launches": 0, "ms": 0.0})
            p["launches"] += rec["launches"]
            p["ms"] += rec["ms"]
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    barrier(world)
    clocks = sampler.stop()
    launches = T.twopaco_kernel_launches() - launches0
    T.twopaco_profile_enable(False)
    run.release_plan()
    st = run.stats(stream)

    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ms, world)
    value = world * m / (ms_max * 1e-3) / 1e9

    # end to end through the host API: pinned host input in, host result out
    pinned = torch.empty(m, dtype=torch.uint8, pin_memory=True)
    pinned.numpy()[:] = bases
    host = pinned.numpy()
    host_seqs = [host[int(off[t]):int(off[t + 1])] for t in range(n)]
    e2e_t = []
    junctions = st["pass2_marks"]
    ctx = T.Context()
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        t0 = time.perf_counter()
        got, est = ctx.build(host_seqs, K, FILTER_BITS, ROUNDS, opts, copy=False)
        if i:
            e2e_t.append(time.perf_counter() - t0)
        assert sum(g.size for g in got) == junctions, "host API and device run disagree"
    ctx.close()
    e2e_s = max_over_ranks(statistics.mean(e2e_t), world) if e2e_t else None
    # served leg: a Poisson stream of build requests through the continuous-batching loop
    served = None
    if args.serve_requests > 0:
        from paper_1602_05856_gb300 import serve
        reqs = serve.served_requests(seqs, args.serve_requests, 20.0, seed=1606)
        slots = [serve.GpuSlot(device=f"cuda:{local}") for _ in range(4)]
        for sl in slots:  # resident buffers sized for the trace, as a server keeps them
            sl.reserve(reqs)
            for r in serve.served_requests(seqs, 2, 1000.0, seed=7):  # both request shapes (k 25, 31)
                serve.run_alone(sl, [r])
        import gc
        gc.collect()
        gc.disable()  # no collector pause inside the timed loops
        try:
            mix = serve.Scheduler(slots, 120 << 30).run(reqs).summary()
            alone_reqs = serve.served_requests(seqs, args.serve_requests, 20.0, seed=1606)
            alone = serve.run_alone(slots[0], alone_reqs).summary()
        finally:
            gc.enable()
        keys = ("p50_ms", "p95_ms", "p99_ms", "max_ms", "throughput_gbps", "wall_s")
        served = {"requests": args.serve_requests, "rate_per_s": 20.0, "slots": 4,
                  "budget_gb": 120,
                  "mix": {k: mix[k] for k in keys},
                  "alone": {k: alone[k] for k in keys},
                  "request_recipe": "2-7 prefixes of the 7 genomes, log-uniform 0.1-5 Mbp, k 25/31, "
                                    "~8 filter bits per base, 4 hashes"}

    batched = batched_leg(T, genomes, dev) if args.batched and rank == 0 else None

    # roofline of the dominant kernel
    table_bytes = st["table_slots"] * (8 if K <= 27 else 16 if K <= 31 else 32)
    # the kernel with the largest share among those with a work model
    modelled = [kv for kv in prof.items() if kernel_work(kv[0], st, m, n, table_bytes)[0] is not None]
    top = max(modelled or prof.items(), key=lambda kv: kv[1]["ms"])
    name, rec = top
    per_launch_ms = rec["ms"] / rec["launches"]
    amount, kind = kernel_work(name, st, m, n, table_bytes)
    if amount is None:
        amount, kind = 0.0, "hbm"
    peaks_json = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = float(peaks_json.get("hbm_gbs", 6800.0))
    if kind == "hbm":
        achieved = amount / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks_json else "fallback 6.8 TB/s"}
    else:
        pk = (l2_read if kind == "l2_read" else l2_or) / 1e9
        achieved = amount / (per_launch_ms * 1e-3) / 1e9
        roof = {"bound": "l2", "achieved": achieved, "peak": pk, "unit": "Gsector/s",
                "frac": achieved / pk if pk > 0 else None, "traffic": None,
                "peak_source": ("measured in this run: random "
                                + ("8-byte loads" if kind == "l2_read" else "64-bit atomic ORs")
                                + f" over a {FILTER_BITS // 8 >> 20} MiB buffer (the filter's size), "
                                "all SMs, best of 5")}
    roof["kernel"] = name
    roof["traffic"] = ncu_traffic(WORKLOAD, name)
    roof["traffic_unit"] = "DRAM bytes per launch (ncu, cold cache)"
    roof["kernel_ms"] = per_launch_ms

    kernels = {k: {"launches": v["launches"], "ms_per_launch": v["ms"] / v["launches"],
                   "share": v["ms"] / sum(x["ms"] for x in prof.values())}
               for k, v in prof.items()}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        sample = sample_prefix(seqs, CPU_SAMPLE_BASES)
        cores = host_cores()
        cpu = {"value": oracle_gbps(sample, K, threads=cores), "unit": UNIT, "cores": cores,
               "kind": "oracle",
               "sample": f"{sum(s.size for s in sample)} bases: the first "
                         f"{sample[0].size} bases of each of the 7 genomes; the definition split "
                         f"over {cores} threads by k-mer hash class",
               "single_thread_value": oracle_gbps(sample, K)}
    lat = sorted(step_ms)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(m) | {"parallelism": f"replicas{world}" if world > 1 else "single"},
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "e2e": {"value": world * m / e2e_s / 1e9, "unit": UNIT,
                "h2d_bytes_per_step": m + 8 * (n + 1),
                "d2h_bytes_per_step": 8 * (n + 1) + 8 * junctions,
                "api": "twopaco_build_ctx: pinned host ASCII in, H2D, run, D2H of offsets and "
                       "positions into pinned memory, on a reused context"} if e2e_s else None,
        "gpu_launches": launches,
        "roofline": roof,
        "cpu_baseline": cpu,
        "served": served,
        "batched": batched,
        "clocks": clocks,
        "stats": {k: st[k] for k in ("positions", "pass1_marks", "pass2_marks", "table_slots")},
        "kernels": kernels,
        "l2_peaks_gsector_s": {"read8": l2_read / 1e9, "or64": l2_or / 1e9, "read32": l2_sector / 1e9},
        "timed_wall_s": wall,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_1602_05856_gb300 import genomes
    import oracle
    seqs = genomes.named_set(WORKLOAD)
    m = sum(s.size for s in seqs)
    sample = sample_prefix(seqs, REF_STEP_BASES)
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
    desc = (f"{sb.size} bases per step: the first {sample[0].size} bases of each of the 7 genomes; "
            f"CPU oracle (plain definition) split over {cores} threads by k-mer hash class")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": workload_config(m) | {"parallelism": "single"},
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
