"""The method's own edge cases on the GPU, against the oracle.

Every other parity input uses the recipe's spectrum (core <= -0.3 Eh, virtual
>= +0.05 Eh, sorted), where every denominator is bounded away from zero. The
regulated small-denominator behaviour is what the DSRG is about (Sec. II.B:
t ~ v s D as D -> 0, so no intruder divergence), so these tests feed inputs
that reach it:

* ``overlap``: virtual energies below core and active ones, unsorted blocks;
  denominators of F1, F2, F3 and the active block cross zero;
* ``degenerate``: the same with planted dyadic energies that make one
  denominator of F1, F2 and F3 exactly zero (the regulator must give 0 there);
* ``negative``: every virtual energy negative (E * eps > 0 in the factorised
  exponentials);
* a flow parameter s = 50, large enough that the factorised exponentials of
  the split epilogues could overflow, so those pairs must take the direct
  expm1 path.

The split kernels count which epilogue branch each work item took
(``dsrg_plan_branch_counts``); the tests assert that the branches meant for
these inputs ran. Bars: FP64 plans 1e-10 relative per block; split plans the
rounding-count bound of the truncating tensor-core accumulator (see
test_gpu_split.py) per block; pair energies element by element.
"""
import math

import numpy as np
import pytest

from dsrg_synth import make_problem
from oracle import dsrg as odsrg

pytestmark = pytest.mark.gpu

BLOCKS = ["ccvv", "cavv", "ccav", "active", "total"]
KSTEP = {"tf32x3": 8, "bf16x3": 16}
LOLO = {"tf32x3": 2.0 ** -24, "bf16x3": 2.0 ** -18}


def bar(prec, naux, block):
    if prec == "fp64":
        return 1e-10
    definite = 1.0 if block == "ccvv" else 2.0
    return definite * 2.0 * (3 * math.ceil(naux / KSTEP[prec]) * 2.0 ** -23 + LOLO[prec])


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    pk.build()
    return pk


def _energy(pk, p, prec):
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec)
    dev = pk.to_device(p)
    plan.branch_counts(reset=True)
    out = plan.energy(*dev, p.s).cpu().numpy()
    cnt = plan.branch_counts(reset=True)
    pairs = plan.pair_energies(dev[0], dev[1], p.s).cpu().numpy()
    plan.sync()
    plan.close()
    return dict(zip(BLOCKS, out)), pairs, cnt


def _compare(gpu, pairs, ref, prec, naux, label):
    for k in BLOCKS:
        rel = abs(gpu[k] - ref[k]) / max(abs(ref[k]), 1e-300)
        print(f"{label} {prec} {k:7s} gpu={gpu[k]:+.15e} oracle={ref[k]:+.15e} rel={rel:.2e}")
        assert rel <= bar(prec, naux, k), (k, rel)
    # pair energies element by element; a pair whose terms cancel is measured
    # against the scale of the largest pair energy
    scale = np.maximum(np.abs(ref["pairs"]), 1e-2 * np.abs(ref["pairs"]).max())
    worst = (np.abs(pairs - ref["pairs"]) / scale).max()
    print(f"{label} {prec} pairs worst {worst:.2e}")
    assert worst <= 2.0 * bar(prec, naux, "ccvv")


EDGE = [
    # spectrum, nC, nA, nV, naux, s, seed: several 128-wide virtual tiles with a
    # ragged last one, naux past the FP32 tail of 32
    ("degenerate", 6, 3, 150, 70, 0.5, 31),
    ("overlap", 5, 2, 260, 90, 0.5, 32),
    ("negative", 4, 2, 140, 60, 0.9, 33),
]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("spectrum,nC,nA,nV,Q,s,seed", EDGE)
def test_edge_spectrum_blocks(pk, prec, spectrum, nC, nA, nV, Q, s, seed):
    p = make_problem(nC, nA, nV, Q, s=s, seed=seed, spectrum=spectrum)
    gpu, pairs, cnt = _energy(pk, p, prec)
    ref = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, nC, nA, nV, with_pairs=True)
    print(spectrum, prec, cnt)
    _compare(gpu, pairs, ref, prec, Q, spectrum)
    if prec == "fp64":
        assert all(v == 0 for v in cnt.values())
        return
    # every epilogue block (32 rows x 16 columns of a work item) took one path
    blocks = cnt["ccvv_far"] + cnt["ccvv_factored"] + cnt["ccvv_direct"]
    assert blocks > 0
    if spectrum in ("degenerate", "overlap", "negative"):
        # denominators within 1/4 of zero: the direct expm1 branch of the CCVV
        # epilogue and the FP64 path of the CAVV epilogue ran
        assert cnt["ccvv_direct"] > 0
        assert cnt["cavv_near"] > 0


def test_degenerate_quadruple_contributes_zero(pk):
    """The planted quadruple (core 0, 1; virtual 0, 1) has D = 0 exactly, so its
    F1 term is 0 whatever its integrals (R(0) = 0, the Maclaurin limit of
    Sec. II.B). The pair energies e_01 and e_10, which contain it, match the
    oracle's in both the FP64 and the split path."""
    p = make_problem(6, 3, 150, 70, s=0.5, seed=31, spectrum="degenerate")
    D = p.eps[0] + p.eps[1] - p.eps[p.ncore + p.nactive] - p.eps[p.ncore + p.nactive + 1]
    assert D == 0.0
    for prec in ("fp64", "bf16x3"):
        gpu, pairs, _ = _energy(pk, p, prec)
        ref = odsrg.ccvv_pair_energies(p.B, p.eps, p.s, p.ncore, p.nactive, p.nvirt,
                                       pairs=[(0, 1), (1, 0)]).numpy()
        for (m, n) in [(0, 1), (1, 0)]:
            assert abs(pairs[m, n] - ref[m, n]) <= bar(prec, p.naux, "ccvv") * abs(ref[m, n])


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
def test_unfactorisable_pairs_large_s(pk, prec):
    """s = 50 with denominators crossing zero: the products of the factorised
    exponentials would leave the FP64 range, so the split epilogues must take
    the direct path for those pairs (CCVV) and (core, active) pairs (CAVV)."""
    p = make_problem(4, 2, 140, 60, s=50.0, seed=34, spectrum="overlap")
    gpu, pairs, cnt = _energy(pk, p, prec)
    ref = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, 4, 2, 140, with_pairs=True)
    print("s=50", prec, cnt)
    _compare(gpu, pairs, ref, prec, p.naux, "s=50")
    if prec != "fp64":
        assert cnt["ccvv_unfactorable"] > 0
        assert cnt["ccvv_factored"] == 0
        assert cnt["ccvv_direct"] > 0
        assert cnt["cavv_unfactorable"] > 0


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("spectrum", ["degenerate", "overlap"])
def test_edge_spectrum_gradient(pk, prec, spectrum):
    """dE/dB, dE/deps, dE/ds where denominators cross zero and vanish exactly:
    at D = 0 the adjoint takes the Maclaurin series of the regulator's
    derivative (Sec. II.B), which the oracle's autograd reproduces through the
    same analytic limit. Bars as in test_gpu_grad.py."""
    p = make_problem(4, 2, 40, 30, s=0.5, seed=35, spectrum=spectrum)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec, grad=True)
    out, dB, de, ds = plan.energy_grad(*pk.to_device(p), p.s)
    plan.sync()
    ref = odsrg.energy_and_grad(p.B, p.eps, p.gamma1, p.lambda2, p.s, p.ncore, p.nactive, p.nvirt)
    dB, de, ds = dB.cpu().numpy(), de.cpu().numpy(), float(ds.cpu()[0])
    errB = np.abs(dB - ref["dB"]).max() / np.abs(ref["dB"]).max()
    erre = np.abs(de - ref["deps"]).max() / np.abs(ref["deps"]).max()
    errs = abs(ds - ref["ds"]) / abs(ref["ds"])
    print(spectrum, prec, "dB %.2e deps %.2e ds %.2e" % (errB, erre, errs))
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert errB < tol and erre < tol and errs < tol
    if spectrum == "degenerate":
        # the planted core orbitals' energies enter D = 0 elements of F1 and F3
        k = [0, 1, p.ncore + p.nactive, p.ncore + p.nactive + 1]
        assert np.all(np.abs(de[k] - ref["deps"][k]) <= tol * np.abs(ref["deps"]).max())
