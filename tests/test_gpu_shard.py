"""One molecule shared by several ranks (dsrg_plan_set_shard), run here as
consecutive shards on one GPU: the partial block energies and gradients of
the shards sum to those of the whole molecule (FP64 and BF16x3 plans). Bar:
1e-13 relative for the energies (the shards add the same partial terms in a
different grouping) and 1e-12 of the largest gradient entry (1e-6 for dB of
split plans, whose tensor-core GEMM sums the ranks' parts in another order)."""
import numpy as np
import pytest

from dsrg_synth import make_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    pk.build()
    return pk


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("world", [2, 3])
def test_shards_sum_to_the_molecule(pk, prec, world):
    p = make_problem(7, 2, 150, 80, s=0.5, seed=51)
    dev = pk.to_device(p)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec, grad=True)
    full = plan.energy(*dev, p.s).cpu().numpy()
    _, dB, de, ds = plan.energy_grad(*dev, p.s)
    gfull = (dB.cpu().numpy(), de.cpu().numpy(), float(ds.cpu()[0]))
    parts, gsum = np.zeros(5), [np.zeros_like(gfull[0]), np.zeros_like(gfull[1]), 0.0]
    for r in range(world):
        plan.set_shard(r, world)
        parts += plan.energy(*dev, p.s).cpu().numpy()
        _, dB, de, ds = plan.energy_grad(*dev, p.s)
        gsum[0] += dB.cpu().numpy()
        gsum[1] += de.cpu().numpy()
        gsum[2] += float(ds.cpu()[0])
    plan.set_shard(0, 1)
    again = plan.energy(*dev, p.s).cpu().numpy()
    plan.sync()
    assert np.array_equal(again, full)          # world = 1 restores the whole molecule
    assert np.all(np.abs(parts - full) <= 1e-13 * np.abs(full))
    # dB of split plans is a tensor-core GEMM of S, whose per-rank parts sum in
    # another rounding order: the split gradient's own bound
    tolB = 1e-12 if prec == "fp64" else 1e-6
    print(prec, world, "dB shards vs whole", np.abs(gsum[0] - gfull[0]).max() / np.abs(gfull[0]).max())
    assert np.abs(gsum[0] - gfull[0]).max() <= tolB * np.abs(gfull[0]).max()
    assert np.abs(gsum[1] - gfull[1]).max() <= 1e-12 * np.abs(gfull[1]).max()
    assert abs(gsum[2] - gfull[2]) <= 1e-12 * abs(gfull[2])


def test_shard_pairs_partition(pk):
    for nC in (1, 5, 24):
        for world in (1, 2, 3, 8):
            got = sorted(pr for r in range(world) for pr in pk.shard_pairs(nC, r, world))
            assert got == [(i, j) for i in range(nC) for j in range(i, nC)]
