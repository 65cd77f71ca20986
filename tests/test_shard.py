"""Host logic of the build split by k-mer class, on the CPU (gloo, world size 2 and 3).

A stand-in run takes the library's place: every position has a partition bin
and a junction flag (seeded, the same on every rank); the leader alone cuts the
bins into classes, and a rank's rounds set the C_final bits of the flagged
positions of its classes only. After ``shard.sharded_build`` every rank must
hold the leader's cut and a C_final equal to all flagged positions: the union
of the disjoint per-class bitmaps, merged by one all-reduce.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class StandInRun:
    """The shard_* surface of twopaco.DeviceBuild over CPU tensors."""

    def __init__(self, m: int, rounds: int, q: int = 64, seed: int = 5):
        import torch
        self.torch = torch
        rng = np.random.default_rng(seed)
        self.m, self.rounds, self.q = m, rounds, q
        self.bins = rng.integers(0, q, size=m)
        self.flags = rng.random(m) < 0.3
        self.cut = torch.zeros(rounds + 1, dtype=torch.int32)
        self.cfinal = torch.zeros((m + 31) // 32, dtype=torch.int32)
        self.rounds_run = []
        self.written = None

    def shard_begin(self, compute_cut: bool) -> None:
        self.cfinal.zero_()
        if compute_cut:  # any ascending cut of [0, q) with non-empty classes
            inner = np.sort(np.random.default_rng(99).choice(np.arange(1, self.q), self.rounds - 1,
                                                               replace=False))
            self.cut[:] = self.torch.tensor([0, *inner.tolist(), self.q], dtype=self.torch.int32)

    def state_tensor(self, which: int):
        from paper_1602_05856_gb300 import twopaco
        return self.cut if which == twopaco.STATE_CUTS else self.cfinal

    def shard_rounds(self, shard: int, n_shards: int) -> None:
        from paper_1602_05856_gb300 import shard as S
        cut = self.cut.numpy()
        bits = np.zeros(self.cfinal.numel() * 32, np.uint8)
        for r in S.owned_rounds(shard, n_shards, self.rounds):
            self.rounds_run.append(r)
            mine = (self.bins >= cut[r]) & (self.bins < cut[r + 1]) & self.flags
            bits[:self.m] |= mine.astype(np.uint8)
        words = np.packbits(bits, bitorder="little").view(np.int32)
        self.cfinal |= self.torch.from_numpy(words.copy())

    def write_output(self) -> None:
        self.written = self.cfinal.clone()


def _worker(rank: int, world: int, port: int, out: str, m: int, rounds: int) -> None:
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1602_05856_gb300 import shard as S
    from tests.test_shard import StandInRun
    dist.init_process_group("gloo", rank=rank, world_size=world)
    run = StandInRun(m, rounds)
    S.sharded_build(run, rank, world, dist)
    want = np.packbits(np.pad(run.flags.astype(np.uint8), (0, run.cfinal.numel() * 32 - m)),
                       bitorder="little").view(np.int32)
    with open(out, "w") as f:
        json.dump({"cut": run.cut.tolist(), "rounds": run.rounds_run,
                   "merged_ok": bool(np.array_equal(run.cfinal.numpy(), want)),
                   "wrote": run.written is not None}, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,rounds", [(2, 2), (2, 5), (3, 7)])
def test_sharded_build_merges_disjoint_classes(tmp_path, world, rounds):
    import torch.multiprocessing as mp
    port = _free_port()
    outs = [str(tmp_path / f"r{r}.json") for r in range(world)]
    ctx = mp.get_context("spawn")
    m = 10_007  # not a multiple of 32: a ragged last word
    procs = [ctx.Process(target=_worker, args=(r, world, port, outs[r], m, rounds)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = [json.load(open(o)) for o in outs]
    assert all(g["merged_ok"] for g in got)
    assert all(g["cut"] == got[0]["cut"] for g in got)  # the leader's cut everywhere
    assert sorted(r for g in got for r in g["rounds"]) == list(range(rounds))
    assert [g["wrote"] for g in got] == [True] + [False] * (world - 1)


def test_owned_rounds_partition_the_classes():
    from paper_1602_05856_gb300 import shard as S
    for rounds in range(1, 20):
        for world in range(1, 9):
            parts = [S.owned_rounds(r, world, rounds) for r in range(world)]
            assert sorted(x for p in parts for x in p) == list(range(rounds))
    with pytest.raises(ValueError):
        S.owned_rounds(2, 2, 4)
