"""The full Table 1 on the GPU: terms J and K (three-body cumulant) and the
off-diagonal Fock block f^(1) (Eqs. (12), (14)) through dsrg_mrpt2_energy_ext
and dsrg_mrpt2_energy_grad_ext, against the oracle.

The inputs add a spin-orbital lambda_{UVW}^{XYZ} (real, Hermitian,
antisymmetric in each triple, spin-conserving) and an off-diagonal Fock block
to the usual synthetic problem. Bars as elsewhere: FP64 plans 1e-10 relative
per block; split plans the rounding-count bound of the truncating tensor-core
accumulator (test_gpu_split.py); gradients 1e-10 (FP64) and 1e-5 (split) of
the largest entry of each array.
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


CASES = [
    # nC, nA, nV, naux, s, seed
    (4, 2, 140, 60, 0.5, 41),
    (3, 4, 70, 45, 0.7, 42),
    (2, 6, 40, 36, 0.4, 43),
    (5, 0, 90, 50, 0.5, 44),   # no active orbitals: only f^(1) singles (term A)
]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("nC,nA,nV,Q,s,seed", CASES)
def test_energy_with_lambda3_and_f1(pk, prec, nC, nA, nV, Q, s, seed):
    p = make_problem(nC, nA, nV, Q, s=s, seed=seed, with_lambda3=nA > 0, with_f1=True)
    plan = pk.Plan(nC, nA, nV, Q, precision=prec)
    dev = pk.to_device(p)
    l3, f1 = pk.extra_to_device(p)
    out = plan.energy(*dev, p.s, lambda3=l3, f1=f1).cpu().numpy()
    base = plan.energy(*dev, p.s).cpu().numpy()
    plan.sync()
    ref = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, nC, nA, nV, with_terms=True,
                       lambda3=p.lambda3, f1=p.f1)
    ref0 = odsrg.energy(p.B, p.eps, p.gamma1, p.lambda2, p.s, nC, nA, nV)
    for k, v in zip(BLOCKS, out):
        if ref[k] == 0.0:   # CAVV and CCAV without active orbitals
            assert v == 0.0, k
            continue
        rel = abs(v - ref[k]) / abs(ref[k])
        print(f"{prec} {nC}/{nA}/{nV}/{Q} {k:7s} gpu={v:+.15e} oracle={ref[k]:+.15e} rel={rel:.2e}")
        assert rel <= bar(prec, Q, k), (k, rel)
    # the extra inputs change only the active block, by J + K + the f^(1) part of A-E
    assert np.array_equal(out[:3], base[:3])
    d_ref = ref["active"] - ref0["active"]
    d_gpu = out[3] - base[3]
    assert d_ref != 0.0
    assert abs(d_gpu - d_ref) <= bar(prec, Q, "active") * abs(ref["active"]), (d_gpu, d_ref)
    if nA >= 2:
        assert ref["terms"]["J"] != 0.0 and ref["terms"]["K"] != 0.0


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("nC,nA,nV,Q,s,seed", [CASES[0], CASES[1], CASES[3]])
def test_gradient_with_lambda3_and_f1(pk, prec, nC, nA, nV, Q, s, seed):
    p = make_problem(nC, nA, nV, Q, s=s, seed=seed, with_lambda3=nA > 0, with_f1=True)
    plan = pk.Plan(nC, nA, nV, Q, precision=prec, grad=True)
    dev = pk.to_device(p)
    l3, f1 = pk.extra_to_device(p)
    out, dB, de, ds = plan.energy_grad(*dev, p.s, lambda3=l3, f1=f1)
    plan.sync()
    ref = odsrg.energy_and_grad(p.B, p.eps, p.gamma1, p.lambda2, p.s, nC, nA, nV,
                                lambda3=p.lambda3, f1=p.f1)
    dB, de, ds = dB.cpu().numpy(), de.cpu().numpy(), float(ds.cpu()[0])
    errB = np.abs(dB - ref["dB"]).max() / np.abs(ref["dB"]).max()
    erre = np.abs(de - ref["deps"]).max() / np.abs(ref["deps"]).max()
    errs = abs(ds - ref["ds"]) / abs(ref["ds"])
    print(prec, nC, nA, nV, Q, "dB %.2e deps %.2e ds %.2e" % (errB, erre, errs))
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert errB < tol and erre < tol and errs < tol
    assert abs(float(out[4].cpu()) - ref["total"]) <= bar(prec, Q, "total") * abs(ref["total"])
