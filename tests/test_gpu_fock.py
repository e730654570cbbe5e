"""Generalized Fock matrix (Eq. (8)) and semicanonicalisation (Sec. III,
steps 2-3) on the GPU against the oracle (oracle/fock.py), and the energy of
the semicanonicalised problem computed from the GPU's outputs against the
oracle's energy of the oracle's semicanonicalised problem.

Everything here is FP64. Bars: f and the orbital energies 1e-12 of the
largest |f|; the transformed factors, f^(1), G', lambda2', lambda3' and U
1e-9 (eigenvectors of well-separated eigenvalues are determined to about
eps_mach ||f|| / gap); the energies 1e-10 relative, the FP64 bar.
"""
import numpy as np
import pytest

from dsrg_synth import make_fock_problem
from oracle import dsrg as odsrg
from oracle import fock as ofock

pytestmark = pytest.mark.gpu

BLOCKS = ["ccvv", "cavv", "ccav", "active", "total"]


@pytest.fixture(scope="module")
def pk():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1603_00561_gb300 as pk
    pk.build()
    return pk


def _dev(x):
    import torch
    return None if x is None else torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64).cuda()


CASES = [
    # nC, nA, nV, naux, seed, with lambda3
    (4, 2, 50, 40, 1, True),
    (3, 3, 100, 70, 2, True),
    (6, 0, 130, 60, 3, False),
    (1, 1, 257, 33, 4, False),   # single core and active orbital; odd virtual count
    (24, 2, 372, 1200, 0, False),  # the cc-pVTZ-sized molecule
]


@pytest.mark.parametrize("nC,nA,nV,Q,seed,l3", CASES)
def test_fock_and_semicanonical_inputs(pk, nC, nA, nV, Q, seed, l3):
    p = make_fock_problem(nC, nA, nV, Q, seed=seed, with_lambda3=l3)
    sc = pk.SemicanonicalPlan(nC, nA, nV, Q)
    h, B, G, L, L3 = (_dev(x) for x in (p.h, p.Bfull, p.gamma1 if nA else None,
                                        p.lambda2 if nA else None, p.lambda3))
    f_gpu = sc.fock(h, B, G).cpu().numpy()
    out = sc.semicanonicalize(h, B, G, L, L3)
    ref = ofock.semicanonicalize(p.h, p.Bfull, p.gamma1, p.lambda2, nC, nA, nV,
                                 p.lambda3 if l3 else None)
    fmax = np.abs(ref["f"]).max()
    print(nC, nA, nV, Q, "Jacobi sweeps", sc.last_sweeps())
    assert np.abs(f_gpu - ref["f"]).max() <= 1e-12 * fmax
    assert np.abs(out["eps"].cpu().numpy() - ref["eps"]).max() <= 1e-12 * fmax
    assert np.abs(out["U"].cpu().numpy() - ref["U"]).max() <= 1e-9
    bmax = np.abs(ref["B"]).max()
    assert np.abs(out["B"].cpu().numpy() - ref["B"]).max() <= 1e-9 * bmax
    assert np.abs(out["f1"].cpu().numpy() - ref["f1"]).max() <= 1e-9 * fmax
    if nA:
        assert np.abs(out["gamma1"].cpu().numpy() - ref["gamma1"]).max() <= 1e-9
        assert np.abs(out["lambda2"].cpu().numpy() - ref["lambda2"]).max() <= 1e-9
    if l3:
        assert np.abs(out["lambda3"].cpu().numpy() - ref["lambda3"]).max() <= 1e-9
    sc.close()


@pytest.mark.parametrize("nC,nA,nV,Q,seed,l3", CASES[:3])
def test_energy_of_the_semicanonicalised_problem(pk, nC, nA, nV, Q, seed, l3):
    """Fock build -> semicanonical inputs -> DSRG-MRPT2 energy with f^(1) (and
    lambda3), all on the GPU, against the same chain in the oracle."""
    p = make_fock_problem(nC, nA, nV, Q, seed=seed, with_lambda3=l3)
    sc = pk.SemicanonicalPlan(nC, nA, nV, Q)
    out = sc.semicanonicalize(_dev(p.h), _dev(p.Bfull), _dev(p.gamma1) if nA else None,
                              _dev(p.lambda2) if nA else None, _dev(p.lambda3))
    plan = pk.Plan(nC, nA, nV, Q, precision="fp64")
    e = plan.energy(out["B"], out["eps"], out["gamma1"], out["lambda2"], p.s,
                    lambda3=out["lambda3"], f1=out["f1"]).cpu().numpy()
    plan.sync()
    r = ofock.semicanonicalize(p.h, p.Bfull, p.gamma1, p.lambda2, nC, nA, nV,
                               p.lambda3 if l3 else None)
    ref = odsrg.energy(r["B"], r["eps"], r["gamma1"], r["lambda2"], p.s, nC, nA, nV,
                       lambda3=r.get("lambda3"), f1=r["f1"])
    for k, v in zip(BLOCKS, e):
        if ref[k] == 0.0:
            assert v == 0.0
            continue
        rel = abs(v - ref[k]) / abs(ref[k])
        print(f"sc {nC}/{nA}/{nV}/{Q} {k:7s} gpu={v:+.15e} oracle={ref[k]:+.15e} rel={rel:.2e}")
        assert rel <= 1e-10, (k, rel)
    sc.close()
