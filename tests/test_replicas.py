"""The multi-process replica path of bench.py on the CPU (gloo, world size 2).

Every rank runs an independent replica (no data-path collective); the bench
joins them only by a barrier and a MAX all-reduce of the step time, and rank 0
alone prints. Exercised here with two gloo processes on 127.0.0.1.
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out: str) -> None:
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_init()
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    got = bench.max_over_ranks(1.0 + rank * 0.5, w)  # rank times 1.0 and 1.5: the max is the job's
    with open(out, "w") as f:
        json.dump({"rank": r, "max": got}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_barrier_and_max_over_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    outs = [str(tmp_path / f"r{r}.json") for r in range(2)]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, outs[r])) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = [json.load(open(o)) for o in outs]
    assert [g["max"] for g in got] == [1.5, 1.5]


def test_reference_arm_prints_on_rank_zero_only():
    """torchrun-style launch of the reference arm: rank 0 prints one line, rank 1 exits 0."""
    port = _free_port()
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2",
               CUDA_VISIBLE_DEVICES="")
    procs = []
    for r in range(2):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c",
                                       "import sys, bench; bench.REF_STEP_BASES = 70_000; "
                                       "sys.argv = ['bench.py', '--impl', 'reference', '--gpus', '2', "
                                       "'--steps', '1', '--warmup', '0']; bench.main()"],
                                      cwd=ROOT, env=e, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    assert all(p.returncode == 0 for p in procs), [o[1][-2000:] for o in outs]
    lines0 = [l for l in outs[0][0].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1][0].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    j = json.loads(lines0[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 2 and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
