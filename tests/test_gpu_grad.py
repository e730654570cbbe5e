"""Gradient of the energy through the C ABI (dsrg_mrpt2_energy_grad).

Checked against (1) the oracle's autograd gradient (tier 1, itself pinned by
central differences of the literal Table 1) on small systems, element by
element, and (2) central finite differences of the GPU FP64 energy at the
cc-pVTZ size on 200 random entries of B plus orbital energies and s, with the
combined bound |g_fd - g| <= 1e-6 |g| + 10 eps_mach |E| / h (the second term is
the rounding floor of a difference quotient of a number of size |E|).

Split-precision plans recompute the CCVV pair blocks in TF32x3 on the tensor
cores and assemble dB as one BF16x3 tensor-core GEMM of the symmetric adjoint
matrix S with B^T, one K stage per TMEM accumulation, summed in FP32 with
round-to-nearest (FP64 regulators and epilogues). Each term of that GEMM
carries the 2^-17 relative error of the BF16 hi + lo representation of S and
B; where a dB entry sums few terms (the small systems) that error is not
averaged down, so against the oracle the bound is 1e-5 of the largest entry
of each array (measured up to 2.5e-6). At the cc-pVTZ size, against the FP64
plan, the bound is the 1e-6 gradient bar (measured 3e-7).
"""
import numpy as np
import pytest

from dsrg_synth import CONFIGS, make_problem
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


SMALL = [(3, 2, 20, 30, 0.5, 0), (4, 1, 33, 17, 0.9, 1), (2, 3, 40, 25, 0.3, 2), (3, 0, 30, 20, 0.5, 3),
         (2, 5, 12, 10, 0.7, 4), (10, 4, 60, 200, 0.5, 0)]


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("nC,nA,nV,Q,s,seed", SMALL)
def test_grad_matches_oracle_autograd(pk, prec, nC, nA, nV, Q, s, seed):
    p = make_problem(nC, nA, nV, Q, s=s, seed=seed)
    plan = pk.Plan(nC, nA, nV, Q, precision=prec, grad=True)
    out, dB, de, ds = plan.energy_grad(*pk.to_device(p), p.s)
    plan.sync()
    ref = odsrg.energy_and_grad(p.B, p.eps, p.gamma1, p.lambda2, p.s, nC, nA, nV)
    dB, de, ds = dB.cpu().numpy(), de.cpu().numpy(), float(ds.cpu()[0])
    sc = np.abs(ref["dB"]).max()
    errB = np.abs(dB - ref["dB"]).max() / sc
    erre = np.abs(de - ref["deps"]).max() / np.abs(ref["deps"]).max()
    errs = abs(ds - ref["ds"]) / abs(ref["ds"])
    print(prec, nC, nA, nV, Q, "dB %.2e deps %.2e ds %.2e" % (errB, erre, errs))
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert errB < tol and erre < tol and errs < tol


def test_grad_finite_differences_vtz(pk):
    p = make_problem(**CONFIGS["naphthyne-vtz-398"])
    import torch
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="fp64", grad=True)
    B, eps, g, l = pk.to_device(p)
    out, dB, de, ds = plan.energy_grad(B, eps, g, l, p.s)
    E = float(out[4])
    dB = dB.cpu().numpy()
    h = 1e-5
    floor = 10 * np.finfo(float).eps * abs(E) / h
    rng = np.random.default_rng(0)
    idx = [tuple(int(rng.integers(0, n)) for n in p.B.shape) for _ in range(200)]
    Bf = B.clone()
    worst = 0.0
    for ix in idx:
        v0 = float(Bf[ix])
        Bf[ix] = v0 + h
        ep = float(plan.energy(Bf, eps, g, l, p.s)[4])
        Bf[ix] = v0 - h
        em = float(plan.energy(Bf, eps, g, l, p.s)[4])
        Bf[ix] = v0
        fd = (ep - em) / (2 * h)
        err = abs(fd - dB[ix])
        worst = max(worst, err / (1e-6 * abs(dB[ix]) + floor))
        assert err <= 1e-6 * abs(dB[ix]) + floor, (ix, fd, dB[ix])
    # orbital energies (a core, the active ones, virtuals) and s
    de = de.cpu().numpy()
    for k in [0, 23, 24, 25, 26, 100, 397]:
        e2 = eps.clone()
        e2[k] += h
        ep = float(plan.energy(B, e2, g, l, p.s)[4])
        e2[k] -= 2 * h
        em = float(plan.energy(B, e2, g, l, p.s)[4])
        fd = (ep - em) / (2 * h)
        assert abs(fd - de[k]) <= 1e-6 * abs(de[k]) + floor, (k, fd, de[k])
    ep = float(plan.energy(B, eps, g, l, p.s + h)[4])
    em = float(plan.energy(B, eps, g, l, p.s - h)[4])
    fd = (ep - em) / (2 * h)
    assert abs(fd - float(ds[0])) <= 1e-6 * abs(float(ds[0])) + floor
    print("worst ratio to tolerance", worst)


def test_autograd_function(pk):
    import torch
    p = make_problem(4, 2, 40, 30, s=0.5, seed=5)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision="fp64", grad=True)
    B, eps, g, l = pk.to_device(p)
    B.requires_grad_(True)
    eps.requires_grad_(True)
    s = torch.tensor(0.5, dtype=torch.float64, device="cuda", requires_grad=True)
    E = pk.energy_total(plan, B, eps, s, g, l)
    (3.0 * E).backward()
    _, dB, de, ds = plan.energy_grad(B.detach(), eps.detach(), g, l, 0.5)
    assert torch.equal(B.grad, 3.0 * dB)
    assert torch.allclose(eps.grad, 3.0 * de, rtol=1e-12, atol=0)
    assert abs(float(s.grad) - 3.0 * float(ds[0])) <= 1e-12 * abs(float(ds[0]))


def test_grad_requires_flag(pk):
    p = make_problem(2, 1, 10, 8, s=0.5, seed=6)
    plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux)
    with pytest.raises(pk.DSRGError):
        plan.energy_grad(*pk.to_device(p), p.s)


@pytest.mark.parametrize("split", ["bf16x3", "tf32x3"])
def test_split_grad_against_fp64_plan_vtz(pk, split):
    """cc-pVTZ size: the gradient of a split plan (tensor-core recompute and
    assembly) against the FP64 plan's, normalised by the largest entry of each
    array, within the 1e-6 gradient bar."""
    p = make_problem(**CONFIGS["naphthyne-vtz-398"])
    dev = pk.to_device(p)
    res = {}
    for prec in ("fp64", split):
        plan = pk.Plan(p.ncore, p.nactive, p.nvirt, p.naux, precision=prec, grad=True)
        out, dB, de, ds = plan.energy_grad(*dev, p.s)
        plan.sync()
        res[prec] = (dB.cpu().numpy(), de.cpu().numpy(), float(ds.cpu()[0]))
        plan.close()
    (b64, e64, s64), (b32, e32, s32) = res["fp64"], res[split]
    errB = np.abs(b32 - b64).max() / np.abs(b64).max()
    erre = np.abs(e32 - e64).max() / np.abs(e64).max()
    errs = abs(s32 - s64) / abs(s64)
    print("vtz %s vs fp64 gradient: dB %.2e deps %.2e ds %.2e" % (split, errB, erre, errs))
    assert errB < 1e-6 and erre < 1e-6 and errs < 1e-6
