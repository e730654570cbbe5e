"""Benchmark of the DF/CD DSRG-MRPT2 energy on GB300.

One step = the whole second-order energy (every block: CCVV, CAVV, CCAV,
active) of one synthetic molecule, inputs resident in HBM. Default workload:
the quintuple-zeta-sized instance (nC=24, nA=2, nV=1214, naux=3400, s=0.5),
whose B (0.86 GB) is larger than L2, in split precision.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision tf32x3|bf16x3|fp64]
    python bench.py --impl reference ...   (the CPU oracle on a bounded sample)

Besides the timed energy step, the JSON line carries two more legs (each
timed with CUDA events after its own warm-up): ``gradient`` (E + dE/dB +
dE/deps + dE/ds at the cc-pVTZ size, FP64 and BF16x3 plans, with the split
gradient's error against the FP64 one; ``--no-grad`` skips it) and ``batch``
(64 molecules of uneven size in one graph-captured call against one-by-one
FP64 plans; ``--with-batch 0`` skips it).

Under torchrun each rank computes its own molecule (weak scaling, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CCVV TFLOP/s and E2 wall time per molecule, split-prec vs FP64 at <=1e-7 Eh"
UNIT = "TFLOP/s"
WORKLOADS = {
    "naphthyne-v5z-1240": dict(ncore=24, nactive=2, nvirt=1214, naux=3400, s=0.5),
    "naphthyne-vtz-398": dict(ncore=24, nactive=2, nvirt=372, naux=1200, s=0.5),
    # a smaller case of the same shape family, for ncu captures (B = 147 MB > L2)
    "profile-16x600": dict(ncore=16, nactive=2, nvirt=600, naux=1700, s=0.5),
    # the small synthetic system (quick runs of the reference arm)
    "tiny-74": dict(ncore=10, nactive=4, nvirt=60, naux=200, s=0.5),
}
# nominal dense rates (TFLOP/s) of the recipe, used to scale the measured BF16 peak
NOMINAL = {"bf16": 2250.0, "tf32": 1100.0, "fp64": 1.25}
# DRAM bytes (read + write) per launch of the CCVV kernel from one ncu capture,
# keyed by (workload, precision, item order); summaries under profiles/. Any
# other combination, or a kernel changed since the capture, reports null.
TRAFFIC = {
    # ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the current CCVV kernel,
    # whole tiles without prefetch (profiles/ccvv_dram_per_order_naphthyne-v5z-1240.md); other
    # codes report null
    ("naphthyne-v5z-1240", "bf16x3", 0): 18808265472 + 3898368,
    ("naphthyne-v5z-1240", "bf16x3", 4): 9346629376 + 3872768,
    ("naphthyne-v5z-1240", "bf16x3", 8): 14072587776 + 3752960,
    ("naphthyne-v5z-1240", "bf16x3", 16): 19147768320 + 3742464,
    ("naphthyne-v5z-1240", "bf16x3", 9): 15875443200 + 3923712,
    ("naphthyne-v5z-1240", "bf16x3", 17): 14867894528 + 3962880,
    ("naphthyne-v5z-1240", "bf16x3", 128): 20477330176 + 3740928,
}


TAIL_Q = 32  # auxiliary functions the split-precision CCVV kernel sums on CUDA cores


def ccvv_flops(nC, nV, Q):
    """Algorithmic flops of the CCVV pair products: nC(nC+1) Q nV^2 (i<=j pairs, full v)."""
    return nC * (nC + 1) * Q * nV * nV


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.remove(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, world, device):
    """The largest value of a per-rank number over all ranks (a timing: the job
    is as slow as its slowest rank). One rank: x itself."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(t, world):
    """Sum of a tensor over all ranks (the partial block energies of a sharded
    molecule: one all-reduce of 5 doubles). One rank: t itself."""
    if world <= 1:
        return t
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput under weak scaling: every rank processes the same
    units (its own molecule), so the job does world * units in `seconds`."""
    return world * units_per_rank / seconds


def run_reference(args, world, rank):
    """The CPU oracle (tier 1, the paper's pair loop) on a bounded sample of
    the same workload: each step computes the CCVV pair energies of a fixed set
    of core pairs (both orders) on the host cores."""
    if rank != 0:
        return
    import torch

    from dsrg_synth import make_problem
    from oracle import dsrg as odsrg
    cfg = WORKLOADS[args.workload]
    p = make_problem(seed=0, **cfg)
    npairs = args.ref_pairs
    sample = []
    for k in range(npairs):
        m = (7 * k) % p.ncore
        n = (5 * k + 3) % p.ncore
        if m == n:
            n = (n + 1) % p.ncore
        sample += [(m, n), (n, m)]
    flops = npairs * 2 * p.naux * p.nvirt * p.nvirt  # algorithmic flops of npairs unordered pairs
    for _ in range(args.warmup if args.warmup < 1 else 1):
        odsrg.ccvv_pair_energies(p.B, p.eps, p.s, p.ncore, p.nactive, p.nvirt, pairs=sample[:2])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        odsrg.ccvv_pair_energies(p.B, p.eps, p.s, p.ncore, p.nactive, p.nvirt, pairs=sample)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    val = flops / t / 1e12
    cores = torch.get_num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, **cfg, "precision": "fp64-cpu"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"CCVV pair energies of {npairs} core pairs (both orders) per step"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(workload, seconds=12.0):
    """Time the oracle's CCVV pair loop on as many core pairs as fit in about
    `seconds` of host time (each pair computed in both orders, as the oracle does)."""
    import torch

    from dsrg_synth import make_problem
    from oracle import dsrg as odsrg
    cfg = WORKLOADS[workload]
    p = make_problem(seed=0, **cfg)
    t0 = time.perf_counter()
    odsrg.ccvv_pair_energies(p.B, p.eps, p.s, p.ncore, p.nactive, p.nvirt, pairs=[(0, 1), (1, 0)])
    per = time.perf_counter() - t0
    npairs = max(1, min(p.ncore * (p.ncore - 1) // 2, int(seconds / max(per, 1e-3))))
    sample = []
    k = 0
    for m in range(p.ncore):
        for n in range(m + 1, p.ncore):
            if k < npairs:
                sample += [(m, n), (n, m)]
                k += 1
    t0 = time.perf_counter()
    odsrg.ccvv_pair_energies(p.B, p.eps, p.s, p.ncore, p.nactive, p.nvirt, pairs=sample)
    dt = time.perf_counter() - t0
    flops = npairs * 2 * p.naux * p.nvirt * p.nvirt
    return {"value": flops / dt / 1e12, "unit": UNIT, "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": f"CCVV pair energies of {npairs} core pairs of {workload} (both orders), "
                      f"{dt:.1f} s"}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_gradient(pk, torch):
    """E + dE/dB + dE/deps + dE/ds at the cc-pVTZ size, per molecule, FP64 and BF16x3
    plans; the energy alone for the ratio; the split gradient's error against the
    FP64 plan's (largest difference over the largest entry, per array)."""
    from dsrg_synth import make_problem
    cfg = WORKLOADS["naphthyne-vtz-398"]
    p = make_problem(seed=0, **cfg)
    dev = pk.to_device(p)
    res = {"workload": "naphthyne-vtz-398"}
    grads = {}
    for prec in ("fp64", "bf16x3"):
        plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec, grad=True)
        out, dB, de, ds = plan.energy_grad(*dev, p.s)
        torch.cuda.synchronize()
        grads[prec] = (dB.clone(), de.clone(), float(ds[0]))
        e0, e1 = _events(torch)
        e0.record()
        for _ in range(3):
            plan.energy_grad(*dev, p.s)
        e1.record()
        torch.cuda.synchronize()
        res[f"{prec}_ms_per_gradient"] = e0.elapsed_time(e1) / 3
        plan.energy(*dev, p.s, out=out)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(3):
            plan.energy(*dev, p.s, out=out)
        e1.record()
        torch.cuda.synchronize()
        res[f"{prec}_ms_per_energy"] = e0.elapsed_time(e1) / 3
        plan.sync()
        plan.close()
    (b64, e64, s64), (b32, e32, s32) = grads["fp64"], grads["bf16x3"]
    res["bf16x3_gradient_over_energy"] = res["bf16x3_ms_per_gradient"] / res["bf16x3_ms_per_energy"]
    res["bf16x3_vs_fp64_rel_err"] = {
        "dB": float((b32 - b64).abs().max() / b64.abs().max()),
        "deps": float((e32 - e64).abs().max() / e64.abs().max()),
        "ds": abs(s32 - s64) / abs(s64)}
    return res


def time_batch(pk, torch, nmol, prec):
    """A batch of nmol molecules of the uneven recipe (seeds 0..nmol-1) in one call,
    against one-by-one FP64 plans."""
    from dsrg_synth import batch_sizes, make_problem
    mols = [make_problem(seed=k, s=0.5, **batch_sizes(k)) for k in range(nmol)]
    dev = [pk.to_device(m) for m in mols]
    flops = sum(ccvv_flops(m.ncore, m.nvirt, m.naux) for m in mols)
    b = pk.Batch([(m.ncore, m.nactive, m.nvirt, m.naux) for m in mols], precision=prec)
    svals = [m.s for m in mols]
    order = b.autotune(dev, svals, reps=1) if prec != "fp64" else None   # setup, not timed
    branches = b.autotune_branches(dev, svals, reps=1)                   # setup, not timed
    out = b.energy(dev, svals)          # captures the graph
    b.energy(dev, svals, out=out)
    torch.cuda.synchronize()
    e0, e1 = _events(torch)
    e0.record()
    for _ in range(3):
        b.energy(dev, svals, out=out)
    e1.record()
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 3 / 1e3
    b.sync()
    # one-by-one FP64 plans (each molecule its own plan and launches)
    plans = [pk.Plan(m.ncore, m.nactive, m.nvirt, m.naux, precision="fp64") for m in mols]
    o64 = [pl.energy(*d, m.s) for pl, d, m in zip(plans, dev, mols)]
    torch.cuda.synchronize()
    e0.record()
    for pl, d, m, o in zip(plans, dev, mols, o64):
        pl.energy(*d, m.s, out=o)
    e1.record()
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    ob = out.cpu().numpy()
    err = max(abs(ob[k][4] - float(o64[k][4])) / abs(float(o64[k][4])) for k in range(nmol))
    res = {"n_mol": nmol, "precision": prec, "item_order": order, "graph_branches": branches,
           "ms_per_batch": tb * 1e3,
           "molecules_per_s": nmol / tb, "aggregate_ccvv_tflops": flops / tb / 1e12,
           "graph_kernel_launches": b.launch_count(),
           "fp64_one_by_one_ms": t64 * 1e3, "fp64_one_by_one_molecules_per_s": nmol / t64,
           "max_rel_err_total_vs_fp64": err}
    b.close()
    for pl in plans:
        pl.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "tf32x3", "fp64"])
    ap.add_argument("--workload", default="naphthyne-v5z-1240", choices=list(WORKLOADS))
    ap.add_argument("--ref-pairs", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: all ranks share ONE molecule (its core pairs dealt "
                         "round-robin, one all-reduce of the 5 block energies per step; strong "
                         "scaling) instead of one molecule per rank (weak scaling)")
    ap.add_argument("--no-grad", action="store_true",
                    help="skip the gradient leg (cc-pVTZ size, FP64 and split plans)")
    ap.add_argument("--with-batch", type=int, default=64, metavar="NMOL",
                    help="molecules of the batch leg (uneven sizes, one call, against "
                         "one-by-one FP64 plans); 0 skips it")
    ap.add_argument("--item-order", type=int, default=None, metavar="CODE",
                    help="fixed CCVV schedule code instead of autotuning it")
    ap.add_argument("--schedule-sweep", action="store_true",
                    help="time the CCVV kernel under every candidate schedule code and exit")
    ap.add_argument("--only", choices=["grad", "batch"], default=None,
                    help="run only the gradient leg, or only the batch leg (64 molecules unless "
                         "--with-batch says otherwise), print its JSON and exit (for profiling)")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1603_00561_gb300 as pk
    from dsrg_synth import make_problem

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    pk.build()
    if args.only == "grad":
        if rank == 0:
            print(json.dumps({"gradient": time_gradient(pk, torch)}), flush=True)
        return
    if args.only == "batch":
        if rank == 0:
            print(json.dumps({"batch": time_batch(pk, torch, args.with_batch or 64, args.precision)}),
                  flush=True)
        return
    cfg = WORKLOADS[args.workload]
    shard = args.shard and world > 1
    # weak scaling: each rank its own molecule of the same size; --shard: one
    # molecule (seed 0) shared by all ranks
    p = make_problem(seed=0 if shard else rank, **cfg)
    prec = args.precision
    try:
        plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec, host_io=True)
    except pk.DSRGError as e:
        if prec == "fp64":
            raise
        print(f"# {prec} unavailable ({e}); measuring fp64", file=sys.stderr)
        prec = "fp64"
        plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec, host_io=True)
    B, eps, g, l = pk.to_device(p)
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    if args.schedule_sweep:
        sweep = {}
        for pf in (0, 4):
            for o in (0, 2 << 1, 4 << 1, 8 << 1, (4 << 1) | 1, (8 << 1) | 1, 64 << 1):
                plan.item_order = (pf << 16) | o
                sweep[(pf << 16) | o] = plan.time_ccvv(B, eps, p.s, reps=3)
        if rank == 0:
            print(json.dumps({"schedule_sweep_ccvv_ms": sweep, "workload": args.workload,
                              "precision": prec}), flush=True)
        plan.close()
        return
    # schedule of the CCVV launch (setup, not timed): autotuned on these inputs, or fixed
    if prec == "fp64":
        item_order = None
    elif args.item_order is not None:
        plan.item_order = args.item_order
        item_order = args.item_order
    else:
        item_order = plan.autotune(B, eps, p.s, reps=2)

    if shard:
        plan.set_shard(rank, world)

    def step():
        plan.energy(B, eps, g, l, p.s, out=out)
        if shard:
            sum_over_ranks(out, world)   # the partial block energies of the ranks

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    launches_per_step = plan.last_launch_count()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    with ClockSampler(local) as cs:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    clocks = cs.summary()
    t_local = e0.elapsed_time(e1) / 1e3 / args.steps
    t_step = max_over_ranks(t_local, world, "cuda")
    energies = out.cpu().numpy().tolist()

    flops = ccvv_flops(p.ncore, p.nvirt, p.naux)
    # weak: every rank did a whole molecule; shard: the ranks did one together
    value = (flops / t_step if shard else job_rate(world, flops, t_step)) / 1e12

    # dominant kernel: the CCVV pair contraction alone, timed with CUDA events on the
    # plan's stream inside the library (planes staged first, one untimed launch)
    nk = max(3, min(args.steps, 10))
    if prec != "fp64":
        t_ccvv = plan.time_ccvv(B, eps, p.s, reps=nk) / 1e3
    else:
        pairs_out = torch.empty((p.ncore, p.ncore), dtype=torch.float64, device="cuda")
        plan.pair_energies(B, eps, p.s, out=pairs_out)
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        k0.record(stream)
        for _ in range(nk):
            plan.pair_energies(B, eps, p.s, out=pairs_out)
        k1.record(stream)
        torch.cuda.synchronize()
        t_ccvv = k0.elapsed_time(k1) / 1e3 / nk
    peaks, peak_kind = load_peaks()
    if prec == "fp64":
        mult, peak = 1, peaks["bf16_tflops"] * NOMINAL["fp64"] / NOMINAL["bf16"]
        peak_note = f"bf16 {peak_kind} peak x nominal fp64/bf16 ratio"
    elif prec == "tf32x3":
        mult, peak = 3, peaks["bf16_tflops"] * NOMINAL["tf32"] / NOMINAL["bf16"]
        peak_note = f"bf16 {peak_kind} peak x nominal tf32/bf16 ratio; achieved counts 3 MMA products over Q >= 32"
    else:
        mult, peak = 3, peaks["bf16_tflops"]
        peak_note = f"bf16 {peak_kind} peak; achieved counts 3 MMA products over Q >= 32"
    # the tensor cores take the auxiliary functions Q >= TAIL_Q; the first TAIL_Q are
    # summed on CUDA cores in the epilogue
    mma_flops = flops if prec == "fp64" else ccvv_flops(p.ncore, p.nvirt, max(p.naux - TAIL_Q, 0))
    achieved = mult * mma_flops / t_ccvv / 1e12
    traffic = TRAFFIC.get((args.workload, prec, item_order))
    roofline = {"bound": "tensor" if prec != "fp64" else "fp64", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "kernel": "ccvv pair contraction", "ccvv_ms": t_ccvv * 1e3,
                "algorithmic_tflops": flops / t_ccvv / 1e12, "peak_source": peak_note}
    if prec != "fp64" and "bf16_tflops_sustained" in peaks:
        # context only: the kernel is timed alone, so `peak` / `frac` use the burst figure;
        # against the seconds-long sustained figure (power cap) the same time reads higher
        sus = peaks["bf16_tflops_sustained"] * (NOMINAL["tf32"] / NOMINAL["bf16"] if prec == "tf32x3" else 1.0)
        roofline["peak_sustained"] = sus
        roofline["frac_of_sustained"] = achieved / sus

    # end to end through the host-buffer entry: H2D of the inputs and D2H of out[5] each step
    Bh = torch.from_numpy(np.ascontiguousarray(p.B)).pin_memory()
    eh = torch.from_numpy(p.eps.copy()).pin_memory()
    gh = torch.from_numpy(np.ascontiguousarray(p.gamma1)).pin_memory()
    lh = torch.from_numpy(np.ascontiguousarray(p.lambda2)).pin_memory()
    oh = torch.zeros(5, dtype=torch.float64).pin_memory()
    plan.energy_host(Bh, eh, gh, lh, p.s, out=oh)
    ne2e = max(3, min(args.steps, 7))
    barrier()
    te2e = []
    for _ in range(ne2e):
        t0 = time.perf_counter()
        plan.energy_host(Bh, eh, gh, lh, p.s, out=oh)   # synchronises (host out)
        te2e.append(time.perf_counter() - t0)
    t_e2e = float(np.median(te2e))
    t_e2e = max_over_ranks(t_e2e, world, "cuda")
    h2d = (Bh.numel() + eh.numel() + gh.numel() + lh.numel()) * 8

    # accuracy against the FP64 GPU path, and its E2 time per molecule
    fp64_cmp = None
    if prec != "fp64" and not args.no_fp64_compare:
        p64 = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="fp64")
        o64 = p64.energy(B, eps, g, l, p.s)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        p64.energy(B, eps, g, l, p.s, out=o64)
        f1.record(stream)
        torch.cuda.synchronize()
        r64 = o64.cpu().numpy()
        # the FP64 CCVV kernel alone against the FP64 peak (no measured FP64 peak: the
        # measured BF16 peak times the nominal FP64/BF16 ratio)
        pairs64 = torch.empty((p.ncore, p.ncore), dtype=torch.float64, device="cuda")
        f2 = torch.cuda.Event(enable_timing=True)
        f3 = torch.cuda.Event(enable_timing=True)
        f2.record(stream)
        p64.pair_energies(B, eps, p.s, out=pairs64)
        f3.record(stream)
        torch.cuda.synchronize()
        t64 = f2.elapsed_time(f3) / 1e3
        pk64 = load_peaks()[0]["bf16_tflops"] * NOMINAL["fp64"] / NOMINAL["bf16"]
        a64 = flops / t64 / 1e12
        fp64_cmp = {"fp64_e2_ms_per_molecule": f0.elapsed_time(f1),
                    "fp64_roofline": {"bound": "fp64", "achieved": a64, "peak": pk64,
                                      "unit": "TFLOP/s", "frac": a64 / pk64,
                                      "kernel": "ccvv pair contraction, FP64 path",
                                      "ccvv_ms": t64 * 1e3,
                                      "peak_source": "bf16 measured peak x nominal fp64/bf16 ratio"},
                    "rel_err_vs_fp64": {k: abs(a - b) / abs(b) if b else abs(a)
                                        for k, a, b in zip(pk.BLOCKS, energies, r64)},
                    "abs_err_vs_fp64_eh": {k: abs(a - b) for k, a, b in zip(pk.BLOCKS, energies, r64)}}
        p64.close()

    extra = {}
    if not args.no_grad:
        extra["gradient"] = time_gradient(pk, torch)
    if args.with_batch > 0:
        extra["batch"] = time_batch(pk, torch, args.with_batch, prec)

    if rank == 0:
        cb = None
        if not args.no_cpu_baseline and world == 1:
            cb = cpu_baseline(args.workload)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "strong" if shard else "weak", "vs_baseline": None,
            "dtype": "f64" if prec == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, **cfg, "precision": prec,
                       "item_order": item_order,
                       "l2": ("inputs larger than L2 (B is %.2f GB, L2 129 MB)" % (p.B.nbytes / 1e9))
                       if p.B.nbytes > 129e6 else "inputs smaller than L2"},
            "e2_ms_per_molecule": t_step * 1e3,
            "energies_eh": dict(zip(pk.BLOCKS, energies)),
            "roofline": roofline,
            "cpu_baseline": cb,
            "e2e": {"value": job_rate(world, flops, t_e2e) / 1e12, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 40,
                    "ms_per_step": t_e2e * 1e3},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clocks,
        }
        if fp64_cmp:
            line.update(fp64_cmp)
        line.update(extra)
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
