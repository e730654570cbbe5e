"""Batched energies (dsrg_mrpt2_energy_batched) of molecules of uneven size.

One persistent tensor-core launch covers the CCVV work of every molecule; the
per-item arithmetic and every reduction order are those of a single-molecule
plan, so the batch must reproduce one plan per molecule bit for bit. The
batch members follow the uneven-size recipe (nC 8-40, nA 2-6, nV 100-600,
naux = 3.2 x basis), scaled down here so the oracle check stays quick.
"""
import numpy as np
import pytest

from dsrg_synth import batch_sizes, make_problem
from oracle import dsrg as odsrg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    pk.build()
    return pk


def _mols(specs):
    return [make_problem(*sp[:4], s=sp[4], seed=sp[5]) for sp in specs]


SPECS = [(3, 2, 140, 60, 0.5, 1), (5, 1, 70, 90, 0.3, 2), (2, 4, 260, 50, 1.0, 3),
         (4, 0, 33, 40, 0.5, 4), (6, 3, 129, 128, 0.7, 5)]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3", "fp64"])
def test_batch_matches_single_plans_bitwise(pk, prec):
    mols = _mols(SPECS)
    batch = pk.Batch([(p.ncore, p.nactive, p.nvirt, p.naux) for p in mols], precision=prec)
    dev = [pk.to_device(p) for p in mols]
    out = batch.energy(dev, [p.s for p in mols]).cpu().numpy()
    batch.sync()
    assert batch.launch_count() > 0
    for m, p in enumerate(mols):
        plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec)
        ref = plan.energy(*dev[m], p.s).cpu().numpy()
        assert np.array_equal(out[m], ref), (m, out[m], ref)


def test_batch_graph_replay_and_recapture(pk):
    mols = _mols(SPECS[:3])
    batch = pk.Batch([(p.ncore, p.nactive, p.nvirt, p.naux) for p in mols], precision="bf16x3")
    dev = [pk.to_device(p) for p in mols]
    a = batch.energy(dev, [p.s for p in mols]).cpu().numpy()
    b = batch.energy(dev, [p.s for p in mols]).cpu().numpy()      # replay
    assert np.array_equal(a, b)
    s2 = [0.25 for _ in mols]                                       # new s: re-capture
    c = batch.energy(dev, s2).cpu().numpy()
    for m, p in enumerate(mols):
        ref = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, 0.25, p.ncore, p.nactive, p.nvirt)
        # the split bound of the total (see test_batch_uneven_recipe_against_oracle)
        tol = 2.0 * 2.0 * (3 * -(-p.naux // 16) * 2.0 ** -23 + 2.0 ** -18)
        rel = abs(c[m][4] - ref["total"]) / abs(ref["total"])
        print(f"re-captured total, molecule {m}: rel vs oracle {rel:.2e} (bound {tol:.1e})")
        assert rel <= tol


def test_batch_uneven_recipe_against_oracle(pk):
    """Molecules drawn from the uneven batch recipe (sizes divided by 4 to keep
    the oracle quick), BF16x3, every block against the oracle."""
    specs = []
    for seed in range(6):
        bs = batch_sizes(seed)
        nC, nA, nV = max(2, bs["ncore"] // 4), bs["nactive"], max(8, bs["nvirt"] // 4)
        specs.append((nC, nA, nV, int(round(3.2 * (nC + nA + nV))), 0.5, seed))
    mols = _mols(specs)
    batch = pk.Batch([(p.ncore, p.nactive, p.nvirt, p.naux) for p in mols], precision="bf16x3")
    out = batch.energy([pk.to_device(p) for p in mols], [p.s for p in mols]).cpu().numpy()
    for m, p in enumerate(mols):
        ref = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, p.ncore, p.nactive, p.nvirt)
        # truncating tensor-core accumulator: < 1 ulp (2^-23) per instruction,
        # 3 instructions per K step of 16, E quadratic in the integrals, and a
        # factor 2 for blocks whose terms are not all of one sign
        tol = 2.0 * (3 * -(-p.naux // 16) * 2.0 ** -23 + 2.0 ** -18)   # + dropped lo*lo
        for k, name in enumerate(["ccvv", "cavv", "ccav", "active", "total"]):
            bar = tol if name == "ccvv" else 2.0 * tol
            if ref[name] == 0.0:
                assert out[m][k] == 0.0
            else:
                rel = abs(out[m][k] - ref[name]) / abs(ref[name])
                print(f"uneven molecule {m} {name:7s} rel vs oracle {rel:.2e} (bound {bar:.1e})")
                assert rel <= bar, (m, name)


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_branches_do_not_change_the_energies(pk, prec):
    """The per-molecule blocks forked into 1, 2 or 4 (of at most 8) concurrent graph branches
    (molecule m on branch m mod K, one GEMM output buffer per branch) give the
    same energies bit for bit; the branch autotuner keeps an allowed K."""
    mols = _mols(SPECS)
    batch = pk.Batch([(p.ncore, p.nactive, p.nvirt, p.naux) for p in mols], precision=prec)
    dev = [pk.to_device(p) for p in mols]
    s = [p.s for p in mols]
    assert batch.branches == 4
    res = {}
    for k in (1, 2, 4):
        batch.branches = k
        res[k] = batch.energy(dev, s).cpu().numpy()
        batch.sync()
    assert np.array_equal(res[1], res[2]) and np.array_equal(res[1], res[4])
    with pytest.raises(pk.DSRGError):
        batch.branches = 3
    k = batch.autotune_branches(dev, s, reps=1)
    assert k in (1, 2, 4) and batch.branches == k
    assert np.array_equal(batch.energy(dev, s).cpu().numpy(), res[1])
    small = pk.Batch([(p.ncore, p.nactive, p.nvirt, p.naux) for p in mols[:3]], precision=prec)
    assert small.branches == 2          # three molecules: at most two buffers
    with pytest.raises(pk.DSRGError):
        small.branches = 4


def test_autotune_cache_is_written_and_applied(pk, tmp_path, monkeypatch):
    """With DSRG_AUTOTUNE_CACHE set, the tuners store their winners under keys of
    GPU, precision and size class; a stored choice is applied without timing."""
    import json
    path = tmp_path / "tune.json"
    monkeypatch.setenv("DSRG_AUTOTUNE_CACHE", str(path))
    p = make_problem(6, 2, 300, 120, s=0.5, seed=7)
    dev = pk.to_device(p)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="bf16x3")
    e0 = plan.energy(*dev, p.s).cpu().numpy()
    code = plan.autotune(dev[0], dev[1], p.s, reps=1)
    data = json.loads(path.read_text())
    keys = [k for k in data if k.startswith("ccvv-schedule|")]
    assert len(keys) == 1 and data[keys[0]] == code and "|bf16x3|" in keys[0]
    # a different stored choice is taken as it is
    other = 9 if code != 9 else 17
    pk.tune_cache_put(path, keys[0], other)
    plan2 = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="bf16x3")
    assert plan2.autotune(dev[0], dev[1], p.s, reps=1) == other
    assert plan2.item_order == other
    assert np.array_equal(plan2.energy(*dev, p.s).cpu().numpy(), e0)
    # batches: the schedule and the branch count
    mols = _mols(SPECS[:4])
    bd = [pk.to_device(m) for m in mols]
    s = [m.s for m in mols]
    batch = pk.Batch([(m.ncore, m.nactive, m.nvirt, m.naux) for m in mols], precision="bf16x3")
    c = batch.autotune(bd, s, reps=1)
    k = batch.autotune_branches(bd, s, reps=1)
    data = json.loads(path.read_text())
    bkeys = {k2.split("|")[0]: v for k2, v in data.items() if k2.startswith("batch")}
    assert bkeys == {"batch-ccvv-schedule": c, "batch-branches": k}
    batch2 = pk.Batch([(m.ncore, m.nactive, m.nvirt, m.naux) for m in mols], precision="bf16x3")
    assert batch2.autotune(bd, s, reps=1) == c and batch2.autotune_branches(bd, s, reps=1) == k
    assert batch2.branches == k
