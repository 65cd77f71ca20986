"""Request loop for junction-detection builds: continuous batching on one GPU.

Requests (sets of strings to build, each with its own k, filter size and
rounds) arrive over time. A request is admitted as soon as an execution slot
is free and the device memory it needs -- its input, its workspace (filter,
pass-2 table, bitmaps) and its output -- fits what the requests in flight
leave of the budget; requests that arrive while others run are admitted as
slots and memory free up, and the work of admitted requests overlaps on the
device (one CUDA stream per slot). A slot takes each request's device
buffers from PyTorch's caching allocator and gives them back when the request
is done, so the budget bounds the device memory of the requests in flight
(the cache reuses the blocks: after the first requests nothing is allocated
from the driver); its page-locked host staging only grows. The loop records
each request's latency (completion minus arrival) and reports p50/p99 and
throughput.

The scheduler (``Scheduler``) holds no GPU code; ``GpuSlot`` runs a request
through the C ABI (``twopaco_run_device``) on the slot's stream; tests drive
the scheduler with a fake slot on the CPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from dataclasses import dataclass, field
from typing import Callable, Deque, Dict, List, Optional, Sequence

import numpy as np

from . import twopaco

dataclasses_replace = dataclasses.replace


@dataclass
class Request:
    rid: int
    seqs: Sequence[np.ndarray]
    k: int
    filter_bits: int
    rounds: int = 1
    hashes: int = 4
    arrival: float = 0.0          # seconds, on the loop's clock
    # filled by the loop
    admitted: Optional[float] = None
    done: Optional[float] = None
    result: Optional[List[np.ndarray]] = None
    stats: Optional[Dict[str, int]] = None

    @property
    def bases(self) -> int:
        return int(sum(int(s.size) for s in self.seqs))

    def positions_upper(self) -> int:
        return int(sum(max(0, int(s.size) - self.k + 1) for s in self.seqs))

    table_slots: int = 0          # pass-2 table reserve; 0 = half a slot per base (grown on overflow)
    digest_only: bool = False     # keep (junctions per string, digest of the positions), not the arrays
    digest: Optional[tuple] = None

    def options(self, stream: int = 0) -> twopaco.Options:
        slots = self.table_slots or max(1 << 16, 1 << int(np.ceil(np.log2(max(self.bases // 2, 1)))))
        return twopaco.Options(hashes=self.hashes, cuda_stream=stream, table_slots=slots)

    def device_bytes(self) -> int:
        """Device memory of one run: input, offsets, workspace, outputs."""
        n = len(self.seqs)
        ws = twopaco.twopaco_workspace_size(self.bases, n, self.k, self.filter_bits, self.rounds,
                                            self.options())
        return self.bases + 8 * (n + 1) + ws + 256 + 8 * (n + 1) + 8 * max(self.positions_upper(), 1)


class Slot:
    """Interface of an execution slot (one request at a time)."""

    def start(self, req: Request) -> None:
        raise NotImplementedError

    def poll(self) -> bool:
        """True once the running request has finished (its result is filled)."""
        raise NotImplementedError

    def held_bytes(self) -> int:
        """Device memory the slot keeps (its buffers survive between requests)."""
        raise NotImplementedError


class GpuSlot(Slot):
    """Runs requests on its own CUDA stream.

    A request's host work -- staging its strings in page-locked memory, waiting
    for its counts, reading back exactly its junctions -- runs on the slot's own
    worker thread, so that the scheduler loop never blocks on one request while
    others finish (numpy copies release the interpreter lock). Its device
    buffers come from PyTorch's caching allocator on the slot's stream and go
    back to it when the request is done; a pass-2 table that overflows is grown
    fourfold and the request run again.
    """

    def __init__(self, device: str = "cuda"):
        import concurrent.futures
        import torch
        self.torch = torch
        self.device = torch.device(device)
        if self.device.index is None:  # the worker thread needs an explicit device
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.Stream(device=self.device)
        self.pinned: Dict[str, "torch.Tensor"] = {}
        self.pool = concurrent.futures.ThreadPoolExecutor(max_workers=1)
        self.future = None
        self.current = 0  # device bytes of the request in flight

    def _grow_pinned(self, name: str, nbytes: int):
        t = self.pinned.get(name)
        if t is None or t.numel() < nbytes:
            t = self.torch.empty(max(nbytes, 1), dtype=self.torch.uint8, pin_memory=True)
            self.pinned[name] = t
        return t

    def held_bytes(self) -> int:
        return int(self.current)

    def reserve(self, reqs: Sequence[Request]) -> None:
        """Grow the page-locked staging for the largest of reqs up front, and run the
        largest once, so that serving them later finds its blocks in the caches."""
        if not reqs:
            return
        big = max(reqs, key=lambda r: r.bases)
        self._grow_pinned("input", big.bases + 8 * (len(big.seqs) + 1))
        self._grow_pinned("out_offsets", 8 * (max(len(r.seqs) for r in reqs) + 1))
        self._grow_pinned("out_positions", 8 * max(big.positions_upper(), 1))
        probe = Request(-1, big.seqs, big.k, big.filter_bits, big.rounds, big.hashes)
        self._serve(probe)

    def start(self, req: Request) -> None:
        self.future = self.pool.submit(self._serve, req)

    def _serve(self, req: Request) -> None:
        torch = self.torch
        torch.cuda.set_device(self.device)
        n, m = len(req.seqs), req.bases
        cap = max(req.positions_upper(), 1)
        off = np.zeros(n + 1, dtype=np.uint64)
        np.cumsum(np.array([s.size for s in req.seqs], dtype=np.uint64), out=off[1:])
        off_at = (m + 15) // 16 * 16
        stream = int(self.stream.cuda_stream)
        slots = req.options().table_slots
        direct = all(is_page_locked(s) for s in req.seqs)
        if not direct:  # page-locked staging of the request's input
            host = self._grow_pinned("input", m + 8 * (n + 1))
            hv = host.numpy()
            if m:
                np.concatenate([np.asarray(s, dtype=np.uint8) for s in req.seqs], out=hv[:m])
        offs_host = self._grow_pinned("offsets", 8 * (n + 1))
        offs_host.numpy()[:8 * (n + 1)] = off.view(np.uint8)
        with torch.cuda.stream(self.stream):
            d_in = torch.empty(off_at + 8 * (n + 1), dtype=torch.uint8, device=self.device)
            if direct:  # every string straight from the page-locked store it is a window of
                for t, sq in enumerate(req.seqs):
                    if sq.size:
                        d_in[int(off[t]):int(off[t + 1])].copy_(torch.from_numpy(sq), non_blocking=True)
            elif m:
                d_in[:m].copy_(host[:m], non_blocking=True)
            d_in[off_at:off_at + 8 * (n + 1)].copy_(offs_host[:8 * (n + 1)], non_blocking=True)
            d_out_off = torch.empty(n + 1, dtype=torch.int64, device=self.device)
            d_out_pos = torch.empty(cap, dtype=torch.int64, device=self.device)
            for attempt in range(4):
                opts = dataclasses_replace(req.options(stream), table_slots=slots)
                ws_bytes = twopaco.twopaco_workspace_size(m, n, req.k, req.filter_bits, req.rounds, opts)
                ws = torch.empty(ws_bytes + 256, dtype=torch.uint8, device=self.device)
                self.current = d_in.numel() + ws.numel() + 8 * (n + 1 + cap)
                ws_ptr = (ws.data_ptr() + 255) // 256 * 256
                twopaco.twopaco_run_device(d_in.data_ptr() if m else 0, d_in.data_ptr() + off_at, n, m,
                                           req.k, req.filter_bits, req.rounds, opts, ws_ptr, ws_bytes,
                                           d_out_off.data_ptr(), d_out_pos.data_ptr(), cap)
                h_off = self._grow_pinned("out_offsets", 8 * (n + 1))[:8 * (n + 1)]
                h_off.copy_(d_out_off.view(torch.uint8), non_blocking=True)
                st = twopaco.twopaco_read_stats(ws_ptr, stream, check=False)  # waits for the run
                if st["rc"] == twopaco.EOVERFLOW and attempt < 3:
                    slots *= 4  # the table was too small for this input: grow it and run again
                    del ws
                    continue
                if st["rc"] != twopaco.OK:
                    raise twopaco.TwopacoError(st["rc"], f"request {req.rid}")
                break
            req.stats = st
            offs = h_off.numpy().view(np.uint64)
            total = int(offs[-1])
            h_pos = self._grow_pinned("out_positions", 8 * max(total, 1))[:8 * total]
            if total:  # exactly the junctions, not the capacity
                h_pos.copy_(d_out_pos[:total].view(torch.uint8), non_blocking=True)
            self.stream.synchronize()
            del d_in, ws, d_out_off, d_out_pos  # back to the cache, on this stream
        self.current = 0
        pos = h_pos.numpy().view(np.uint64)
        if req.digest_only:
            req.digest = result_digest(offs, pos)
        else:
            req.result = [pos[offs[t]:offs[t + 1]].copy() for t in range(n)]

    def poll(self) -> bool:
        if self.future is None or not self.future.done():
            return False
        f, self.future = self.future, None
        f.result()  # a failed request raises here
        return True


@dataclass
class ServeReport:
    requests: List[Request] = field(default_factory=list)
    wall_s: float = 0.0

    def latencies(self) -> np.ndarray:
        return np.array([r.done - r.arrival for r in self.requests], dtype=np.float64)

    def summary(self) -> Dict[str, float]:
        lat = self.latencies()
        bases = sum(r.bases for r in self.requests)
        return {"requests": len(self.requests),
                "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else 0.0,
                "p95_ms": float(np.percentile(lat, 95) * 1e3) if lat.size else 0.0,
                "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else 0.0,
                "max_ms": float(lat.max() * 1e3) if lat.size else 0.0,
                "mean_ms": float(lat.mean() * 1e3) if lat.size else 0.0,
                "throughput_gbps": bases / self.wall_s / 1e9 if self.wall_s > 0 else 0.0,
                "wall_s": self.wall_s}


class Scheduler:
    """Admit requests in arrival order as slots and the memory budget allow."""

    def __init__(self, slots: Sequence[Slot], budget_bytes: int,
                 clock: Callable[[], float] = time.perf_counter):
        self.slots = list(slots)
        self.budget = int(budget_bytes)
        self.clock = clock
        self.busy: Dict[int, Request] = {}   # slot index -> request
        self.reserved: Dict[int, int] = {}   # slot index -> bytes reserved

    def free_bytes(self) -> int:
        return self.budget - sum(self.reserved.values())

    def run(self, requests: Sequence[Request], sleep: Callable[[float], None] = time.sleep,
            poll_interval: float = 50e-6) -> ServeReport:
        pending: Deque[Request] = collections.deque(sorted(requests, key=lambda r: r.arrival))
        for r in pending:
            if r.device_bytes() > self.budget:
                raise ValueError(f"request {r.rid} needs more than the whole budget")
        finished: List[Request] = []
        t0 = self.clock()
        while pending or self.busy:
            now = self.clock() - t0
            for i, slot in enumerate(self.slots):
                if i in self.busy and slot.poll():
                    req = self.busy.pop(i)
                    req.done = self.clock() - t0
                    self.reserved.pop(i, None)
                    finished.append(req)
            # admit in arrival order (no overtaking): continuous batching
            while pending and pending[0].arrival <= now:
                free = [i for i in range(len(self.slots)) if i not in self.busy]
                need = pending[0].device_bytes()
                if not free or need > self.free_bytes():
                    break
                i = free[0]
                req = pending.popleft()
                req.admitted = self.clock() - t0
                self.reserved[i] = need
                self.busy[i] = req
                self.slots[i].start(req)
            if not self.busy and pending and pending[0].arrival > now:
                sleep(min(pending[0].arrival - now, 1e-3))
            elif self.busy:
                sleep(poll_interval)
        return ServeReport(finished, self.clock() - t0)


def result_digest(offs: np.ndarray, pos: np.ndarray) -> tuple:
    """(junctions per string, an order-dependent digest of the positions) of one result."""
    counts = tuple(int(x) for x in np.diff(offs.astype(np.int64)))
    with np.errstate(over="ignore"):
        x = pos.astype(np.uint64) ^ (np.arange(pos.size, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15))
        x ^= x >> np.uint64(30)
        x *= np.uint64(0xBF58476D1CE4E5B9)
        x ^= x >> np.uint64(27)
        x *= np.uint64(0x94D049BB133111EB)
        x ^= x >> np.uint64(31)
        return counts, int(x.sum(dtype=np.uint64)) if x.size else 0


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a seeded Poisson stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def served_requests(pool: Sequence[np.ndarray], n: int, rate_per_s: float, seed: int,
                    genomes_range=(2, 7), mbp_range=(0.1, 5.0), ks=(25, 31),
                    bits_per_base: float = 8.0, hashes: int = 4, digest_only: bool = False) -> List[Request]:
    """A seeded stream of build requests over a pool of related genomes.

    Each request takes a number of strings uniform in ``genomes_range``: windows
    of pool genomes at uniform offsets whose lengths are log-uniform in
    ``mbp_range`` (Mbp); k alternates over ``ks``; the filter has about
    ``bits_per_base`` bits per base (a power of two); arrivals are Poisson.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    arrivals = poisson_arrivals(n, rate_per_s, seed + 1)
    out = []
    lo, hi = np.log(mbp_range[0] * 1e6), np.log(mbp_range[1] * 1e6)
    for i in range(n):
        g = int(rng.integers(genomes_range[0], genomes_range[1] + 1))
        seqs = []
        for _ in range(g):
            src = pool[int(rng.integers(0, len(pool)))]
            ln = int(min(src.size, np.exp(rng.uniform(lo, hi))))
            start = int(rng.integers(0, src.size - ln + 1))
            seqs.append(np.ascontiguousarray(src[start:start + ln]))
        bases = sum(s.size for s in seqs)
        bits = 1 << max(8, int(np.ceil(np.log2(bits_per_base * bases))))
        out.append(Request(i, seqs, int(ks[i % len(ks)]), bits, hashes=hashes,
                           arrival=float(arrivals[i]), digest_only=digest_only))
    return out


# The served configuration: 2-50 genomes of 0.1-50 Mbp (log-uniform) per request,
# k 25 or 31, Poisson arrivals at 20 per second, a 120 GB admission budget.
SERVED_GENOMES, SERVED_MBP, SERVED_RATE, SERVED_BUDGET = (2, 50), (0.1, 50.0), 20.0, 120 << 30


_LOCKED: List[np.ndarray] = []


def page_lock(arrays: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Page-lock host arrays in place (cudaHostRegister), as a server keeps its genome
    store, so that windows of them copy to the device without staging. They stay locked
    (and referenced) for the life of the process."""
    import torch
    rt = torch.cuda.cudart()
    out = []
    for a in arrays:
        a = np.ascontiguousarray(a)
        if a.size and rt.cudaHostRegister(a.ctypes.data, a.nbytes, 0) == 0:
            _LOCKED.append(a)
        out.append(a)
    return out


def is_page_locked(a: np.ndarray) -> bool:
    """a lies inside an array page_lock registered (a window of it, e.g.)."""
    if not a.size:
        return True
    p = a.__array_interface__["data"][0]
    return any(b.ctypes.data <= p and p + a.nbytes <= b.ctypes.data + b.nbytes for b in _LOCKED)


def served_pool(lock: bool = False):
    """The genome pool of the served configuration: the bacterial-set recipe at ten
    times its length (7 related genomes of 46-56 Mbp), so that a window can reach 50 Mbp;
    with lock, page-locked as a server's resident store."""
    from . import genomes
    pool = genomes.named_set("bacterial_set", 10.0)
    return page_lock(pool) if lock else pool


def run_alone(slot: Slot, requests: Sequence[Request],
              clock: Callable[[], float] = time.perf_counter) -> ServeReport:
    """Each request by itself on one slot, back to back (latency = its own run)."""
    done = []
    t0 = clock()
    for r in requests:
        a = clock()
        slot.start(r)
        while not slot.poll():
            time.sleep(20e-6)  # let a slot's worker thread run
        r.arrival, r.admitted, r.done = a - t0, a - t0, clock() - t0
        done.append(r)
    return ServeReport(done, clock() - t0)
