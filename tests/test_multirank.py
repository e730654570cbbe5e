"""The multi-rank paths on CPU with the gloo backend (world size 2).

Under torchrun every rank computes its own molecule by default (weak scaling,
no data-path collective); the only collective is the max-over-ranks reduction
of the step times, and the reference arm runs on rank 0 alone. With
``--shard`` the ranks share one molecule: rank r takes the core pairs the
library deals to it (dsrg_shard_pairs) and rank 0 the other blocks, and one
all-reduce of 5 doubles sums the partial block energies. These host-side
pieces are checked here without a GPU: the pair deal partitions the pairs, and
partial energies computed by the oracle on each rank's pairs sum, through the
same reduction bench.py uses, to the oracle's full energy."""
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


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    from dsrg_synth import make_problem
    from oracle import dsrg as odsrg
    from paper_1603_00561_gb300 import shard_pairs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = make_problem(6, 2, 20, 30, s=0.5, seed=17)
    mine = shard_pairs(p.ncore, rank, world)
    # this rank's share: F1 over its pairs (both orders), the other blocks on rank 0
    sym = [(i, j) for (i, j) in mine] + [(j, i) for (i, j) in mine if i != j]
    e = odsrg.ccvv_pair_energies(p.B, p.eps, p.s, p.ncore, p.nactive, p.nvirt, pairs=sym)
    part = torch.zeros(5, dtype=torch.float64)
    part[0] = float(e.sum())
    if rank == 0:
        full = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, p.ncore, p.nactive, p.nvirt)
        part[1], part[2], part[3] = full["cavv"], full["ccav"], full["active"]
    part[4] = part[:4].sum()
    tot = bench.sum_over_ranks(part, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, mine, tot.tolist()))


def test_pair_shards_sum_to_the_energy_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from dsrg_synth import make_problem
    from oracle import dsrg as odsrg
    p = make_problem(6, 2, 20, 30, s=0.5, seed=17)
    full = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, p.ncore, p.nactive, p.nvirt)
    all_pairs = [pr for _, mine, _ in res for pr in mine]
    assert sorted(all_pairs) == [(i, j) for i in range(6) for j in range(i, 6)]
    assert len(set(all_pairs)) == len(all_pairs)
    for _, _, tot in res:
        for k, name in enumerate(["ccvv", "cavv", "ccav", "active", "total"]):
            assert abs(tot[k] - full[name]) <= 1e-12 * abs(full[name]), name


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
