"""Work-item shapes of the split CCVV kernel: every virtual tile whole (N up to
128) or as two column halves (N up to 64; schedule code bit 24; a tile of at
most 64 columns is then one half item). The energy is kept per 64-column
half of every (pair, tile pair), summed in the same order in both shapes, so
the energies (and the gradient's dB) are bitwise the same for every shape and
item order; against the oracle the split bound of tests/test_gpu_split.py holds
as for the default."""
import math

import numpy as np
import pytest

from dsrg_synth import make_problem
from oracle import dsrg as odsrg

pytestmark = pytest.mark.gpu

HALVES = 1 << 24
KSTEP = {"tf32x3": 8, "bf16x3": 16}
LOLO = {"tf32x3": 2.0 ** -24, "bf16x3": 2.0 ** -18}
BLOCKS = ["ccvv", "cavv", "ccav", "active", "total"]


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    pk.build()
    return pk


# nV 300: tiles of 128, 128 and 44 columns; nV 200: 128 and 72; nV 60: one of 60
CASES = [(6, 2, 300, 130, 0.5, 1), (5, 0, 200, 90, 0.9, 2), (3, 3, 60, 70, 0.3, 3),
         (9, 2, 257, 200, 1.0, 4)]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("nC,nA,nV,Q,s,seed", CASES)
def test_shapes_give_bitwise_equal_energies(pk, prec, nC, nA, nV, Q, s, seed):
    p = make_problem(nC, nA, nV, Q, s=s, seed=seed)
    dev = pk.to_device(p)
    plan = pk.Plan(nC, nA, nV, Q, precision=prec)
    res = {}
    for code in (0, HALVES, 9, 9 | HALVES, 8 | HALVES):
        plan.item_order = code
        assert plan.item_order == code
        res[code] = plan.energy(*dev, p.s).cpu().numpy()
    plan.sync()
    for code, e in res.items():
        assert np.array_equal(e, res[0]), (code, e, res[0])
    ref = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, nC, nA, nV)
    rel = abs(res[HALVES][0] - ref["ccvv"]) / abs(ref["ccvv"])
    tol = 2.0 * (3 * math.ceil(Q / KSTEP[prec]) * 2.0 ** -23 + LOLO[prec])
    assert rel <= tol, (rel, tol)


def test_shapes_in_batches_and_the_host_entry(pk):
    mols = [make_problem(*c[:4], s=c[4], seed=c[5]) for c in CASES]
    dev = [pk.to_device(m) for m in mols]
    s = [m.s for m in mols]
    batch = pk.Batch([(m.ncore, m.nactive, m.nvirt, m.naux) for m in mols], precision="bf16x3")
    batch.item_order = 0
    a = batch.energy(dev, s).cpu().numpy()
    batch.item_order = 17 | HALVES
    b = batch.energy(dev, s).cpu().numpy()
    batch.sync()
    assert np.array_equal(a, b)
    # the host-buffer entry runs the items in groups of core rows
    p = mols[0]
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="bf16x3", host_io=True)
    plan.item_order = 4 | HALVES
    eh = plan.energy_host(p.B, p.eps, p.gamma1, p.lambda2, p.s)
    assert np.array_equal(np.asarray(eh), a[0])


def test_shapes_give_the_same_gradient(pk):
    p = make_problem(6, 2, 300, 130, s=0.5, seed=11)
    dev = pk.to_device(p)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="bf16x3", grad=True)
    plan.item_order = 0
    _, dB0, de0, ds0 = plan.energy_grad(*dev, p.s)
    dB0, de0, ds0 = dB0.cpu().numpy(), de0.cpu().numpy(), float(ds0.cpu()[0])
    plan.item_order = HALVES
    _, dB1, de1, ds1 = plan.energy_grad(*dev, p.s)
    plan.sync()
    assert np.array_equal(dB1.cpu().numpy(), dB0)
    # the eps / s derivatives are summed with atomics: equal to rounding
    assert np.abs(de1.cpu().numpy() - de0).max() <= 1e-13 * np.abs(de0).max()
    assert abs(float(ds1.cpu()[0]) - ds0) <= 1e-13 * abs(ds0)
