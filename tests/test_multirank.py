"""The multi-rank path of bench.py on CPU with the gloo backend (world size 2).

Under torchrun every rank computes its own molecule (weak scaling, no
data-path collective); the only collective is the max-over-ranks reduction of
the step times, and the reference arm runs on rank 0 alone. These are the
pieces checked here, without a GPU."""
import json
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_init()
    t = bench.max_over_ranks(1.0 + 2.0 * r, w, "cpu")   # rank 1 is the slow one
    rate = bench.job_rate(w, 10.0, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, t, rate))


def test_max_over_ranks_and_weak_scaling_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, t, rate in res:
        assert w == 2
        assert t == 3.0                  # max over ranks, the same on every rank
        assert rate == 2 * 10.0 / 3.0    # whole-job units over the slowest rank's time


def test_reference_arm_runs_on_rank0_only(capsys):
    import bench

    class A:
        workload = "tiny-74"
        ref_pairs = 2
        steps = 1
        warmup = 0
    bench.run_reference(A, world=2, rank=1)
    assert capsys.readouterr().out == ""
    bench.run_reference(A, world=2, rank=0)
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
