"""The request loop: admission and ordering on the CPU, result identity on the GPU."""
import numpy as np
import pytest

from paper_1602_05856_gb300 import genomes
from paper_1602_05856_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


class FakeSlot(serve.Slot):
    """Finishes a request a fixed time after it started (time per base)."""

    def __init__(self, clock, per_base):
        self.clock, self.per_base, self.req, self.until = clock, per_base, None, 0.0

    def start(self, req):
        self.req, self.until = req, self.clock() + req.bases * self.per_base
        req.result = [np.zeros(0, np.uint64)]

    def poll(self):
        if self.req is not None and self.clock() >= self.until:
            self.req = None
            return True
        return False

    def held_bytes(self):
        return 0


def _requests(n, seed, lo=2000, hi=20000):
    rng = np.random.default_rng(seed)
    arrivals = serve.poisson_arrivals(n, 20.0, seed)
    out = []
    for i in range(n):
        seqs = genomes.random_strings(seed + i, int(rng.integers(1, 4)), lo, hi)
        out.append(serve.Request(i, seqs, 25, 1 << 16, arrival=float(arrivals[i])))
    return out


def test_requests_admitted_in_order_within_budget():
    clock = FakeClock()
    slots = [FakeSlot(clock, 1e-6) for _ in range(3)]
    reqs = _requests(40, 3)
    budget = max(r.device_bytes() for r in reqs) * 2  # at most two requests fit at once
    sched = serve.Scheduler(slots, budget, clock=clock)
    peak = [0]
    orig_start = FakeSlot.start

    def tracking_start(self, req):
        peak[0] = max(peak[0], sum(sched.reserved.values()))
        orig_start(self, req)

    FakeSlot.start = tracking_start
    try:
        rep = sched.run(reqs, sleep=clock.sleep)
    finally:
        FakeSlot.start = orig_start
    assert len(rep.requests) == 40
    assert peak[0] <= budget
    admitted = sorted(rep.requests, key=lambda r: r.admitted)
    assert [r.rid for r in admitted] == sorted(r.rid for r in reqs)  # no overtaking
    assert all(r.admitted >= r.arrival and r.done >= r.admitted for r in rep.requests)
    s = rep.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_request_larger_than_budget_is_refused():
    clock = FakeClock()
    reqs = _requests(2, 5)
    sched = serve.Scheduler([FakeSlot(clock, 1e-6)], budget_bytes=1024, clock=clock)
    with pytest.raises(ValueError):
        sched.run(reqs, sleep=clock.sleep)


@pytest.mark.gpu
def test_each_result_is_the_same_alone_and_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from paper_1602_05856_gb300 import build, twopaco as T
    build.build()
    base = genomes.named_set("plain_single", 0.05)
    rng = np.random.default_rng(11)
    reqs = []
    arrivals = serve.poisson_arrivals(24, 200.0, 7)
    for i in range(24):
        pick = [base[j][: int(rng.integers(5000, base[j].size))] for j in range(int(rng.integers(1, 5)))]
        k = [15, 25, 31, 63][i % 4]
        reqs.append(serve.Request(i, pick, k, 1 << int(rng.integers(16, 22)), rounds=1 + (i % 3 == 0),
                                  hashes=3 + i % 4, arrival=float(arrivals[i])))
    slots = [serve.GpuSlot() for _ in range(3)]
    rep = serve.Scheduler(slots, budget_bytes=8 << 30).run(reqs)
    assert len(rep.requests) == 24
    for r in rep.requests:
        alone, _ = T.twopaco_build_ex(r.seqs, r.k, r.filter_bits, r.rounds,
                                      T.Options(hashes=r.hashes))
        assert all(np.array_equal(a, b) for a, b in zip(alone, r.result)), r.rid
        if r.rid % 6 == 0:
            want = O.junctions(genomes.concat(r.seqs), r.k)
            assert all(np.array_equal(a, b) for a, b in zip(want, r.result)), r.rid
    assert rep.summary()["p99_ms"] > 0


@pytest.mark.gpu
def test_served_recipe_same_alone_in_the_mix_and_by_definition():
    """Requests of the served configuration (2-50 windows of 0.1-50 Mbp from the 10x
    bacterial pool, k 25/31) arriving faster than they finish, over 3 slots under the
    120 GB budget: every result equals the request run alone, and the smaller ones equal
    the oracle's junctions."""
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from paper_1602_05856_gb300 import build
    build.build()
    pool = serve.served_pool(lock=True)
    assert all(serve.is_page_locked(g) for g in pool) and serve.is_page_locked(pool[0][10:1000])
    reqs = serve.served_requests(pool, 10, 200.0, seed=2024, genomes_range=serve.SERVED_GENOMES,
                                 mbp_range=serve.SERVED_MBP)
    slots = [serve.GpuSlot() for _ in range(3)]
    rep = serve.Scheduler(slots, serve.SERVED_BUDGET).run(reqs)
    assert len(rep.requests) == 10
    alone = serve.served_requests(pool, 10, 200.0, seed=2024, genomes_range=serve.SERVED_GENOMES,
                                  mbp_range=serve.SERVED_MBP)
    serve.run_alone(slots[0], alone)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    checked = 0
    for r, a in zip(sorted(rep.requests, key=lambda x: x.rid), alone):
        assert all(np.array_equal(x, y) for x, y in zip(r.result, a.result)), r.rid
        if r.bases <= 120_000_000 and checked < 2:
            want = O.junctions(genomes.concat(r.seqs), r.k, threads=cores)
            assert all(np.array_equal(x, y) for x, y in zip(want, r.result)), r.rid
            checked += 1
    assert checked >= 1


def test_result_digest_tells_results_apart():
    o = np.array([0, 3, 5], np.uint64)
    a = serve.result_digest(o, np.array([1, 2, 3, 7, 9], np.uint64))
    assert a == serve.result_digest(o, np.array([1, 2, 3, 7, 9], np.uint64))
    assert a != serve.result_digest(o, np.array([1, 2, 3, 9, 7], np.uint64))  # order counts
    assert a != serve.result_digest(o, np.array([1, 2, 3, 7, 10], np.uint64))
    assert a != serve.result_digest(np.array([0, 2, 5], np.uint64), np.array([1, 2, 3, 7, 9], np.uint64))
