"""Schedule autotuning of the split-precision CCVV launch.

The order in which work items are dealt to the SMs, and how far ahead the
producer prefetches operand tiles into L2, decide which tiles share the L2 at
any moment, but not the result: every item writes its
own partial sum, and the partials are reduced in a fixed order. So every
candidate order must give bit-for-bit the same energies, and the autotuner
must pick one of the candidates."""
import numpy as np
import pytest

from dsrg_synth import batch_sizes, make_problem

pytestmark = pytest.mark.gpu

ORDERS = {0, 2 << 1, 4 << 1, 8 << 1, (4 << 1) | 1, (8 << 1) | 1, 64 << 1}
# prefetch 0, 4 or 12 K stages; without prefetch also every tile in column halves (bit 24)
CANDIDATES = {(pf << 16) | o for pf in (0, 4, 12, 1 << 8) for o in ORDERS}


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    pk.build()
    return pk


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_plan_orders_bitwise_and_autotune(pk, prec):
    p = make_problem(11, 2, 300, 150, s=0.5, seed=31)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec)
    dev = pk.to_device(p)
    ref = plan.energy(*dev, p.s).cpu().numpy()
    ref_pairs = plan.pair_energies(dev[0], dev[1], p.s).cpu().numpy()
    for order in sorted(ORDERS) + [(3 << 1) | 1, (8 << 16) | (4 << 1), (64 << 16) | 1]:
        plan.item_order = order
        assert plan.item_order == order
        assert np.array_equal(plan.energy(*dev, p.s).cpu().numpy(), ref), order
        assert np.array_equal(plan.pair_energies(dev[0], dev[1], p.s).cpu().numpy(), ref_pairs), order
    chosen = plan.autotune(dev[0], dev[1], p.s, reps=2)
    assert chosen in CANDIDATES and plan.item_order == chosen
    assert np.array_equal(plan.energy(*dev, p.s).cpu().numpy(), ref)
    ms = plan.time_ccvv(dev[0], dev[1], p.s, reps=3)
    assert 0.0 < ms < 1e4
    plan.sync()


def test_fp64_plan_autotune_is_noop(pk):
    p = make_problem(3, 1, 40, 20, s=0.5, seed=32)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="fp64")
    dev = pk.to_device(p)
    assert plan.autotune(dev[0], dev[1], p.s) == -1
    assert plan.item_order == -1
    with pytest.raises(pk.DSRGError):
        plan.time_ccvv(dev[0], dev[1], p.s)


def test_batch_autotune_bitwise(pk):
    mols = []
    for seed in range(5):
        bs = batch_sizes(seed)
        nC, nA, nV = max(2, bs["ncore"] // 3), bs["nactive"], max(8, bs["nvirt"] // 3)
        mols.append(make_problem(nC, nA, nV, int(round(3.2 * (nC + nA + nV))), s=0.5, seed=seed))
    batch = pk.Batch([(p.ncore, p.nactive, p.nvirt, p.naux) for p in mols], precision="bf16x3")
    dev = [pk.to_device(p) for p in mols]
    svals = [p.s for p in mols]
    ref = batch.energy(dev, svals).cpu().numpy()
    chosen = batch.autotune(dev, svals, reps=1)
    assert chosen in CANDIDATES and batch.item_order == chosen
    assert np.array_equal(batch.energy(dev, svals).cpu().numpy(), ref)
    batch.item_order = (2 << 1) | 1
    assert np.array_equal(batch.energy(dev, svals).cpu().numpy(), ref)
    batch.sync()
