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
        assert abs(c[m][4] - ref["total"]) / abs(ref["total"]) <= tol


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
                assert abs(out[m][k] - ref[name]) / abs(ref[name]) <= bar, (m, name)
